// fempic_env.cu -- sm_103a kernels and the C ABI of the envelope-tracking
// FEMPIC particle step (include/fempic_env.h).
//
// Data layout on the device (per tet, indexed by tet id):
//   geom64  double[12]  x0, grad l1, grad l2, grad l3        (96 B, FP64 form + location)
//   tetrec  float4 x8   mixed form, one 128 B line per tet: x0 as an FP32 pair
//                       and grad l1..l3 (64 B), the per-step affine field
//                       (48 B, written by k_field_f32), neighbours (16 B)
//   tn      int4        sorted global node ids
//   nb      int4        neighbour across local face k, or wall code
//   te      int4 x 2    6 global edge ids, padded to 8
//   tf      int4        4 global face ids
//   field   per step: the affine envelope field of the tet after the carrier
//           is restored, E(r) = E0 + (r - x0) x W, B(r) = B0 + beta (r - x0):
//           double[10] (FP64 form) or float[12] (mixed form).
// Whitney-1 fields are affine with an antisymmetric gradient and Whitney-2
// fields are affine with an isotropic gradient, so these 10 numbers carry the
// whole gather of Sec. III-A for every particle in the tet; they are built
// once per step from the 10 complex DoFs of the tet by k_field_*.
//
// Particle SoA (caller owned): x, y, z f64; vx, vy, vz f64 (FP64 form) or f32
// (mixed); tet i32; status u8; n_cross i32 (optional).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "fempic_internal.h"

using namespace fempic;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define FEMPIC_CUDA(call)                                                                      \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail(FEMPIC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));           \
  } while (0)

constexpr int kThreads = 256;
constexpr int kQBits = 24;                       // fixed-point barycentrics of the mixed form
constexpr float kQScale = 16777216.0f;           // 2^24
constexpr int32_t kQOne = 1 << kQBits;
constexpr float kQClamp = 32.0f;
constexpr int32_t kMaxCrossingsLimit = 1 << 20;

// Local topology of a tet with sorted nodes, usable in device code: edge e
// joins (le0(e), le1(e)) in the order 01,02,03,12,13,23; face f is opposite
// node f and its i-th node (ascending) is lf(f, i).
__host__ __device__ constexpr int le0(int e) { return e < 3 ? 0 : (e < 5 ? 1 : 2); }
__host__ __device__ constexpr int le1(int e) { return e < 3 ? e + 1 : (e == 3 ? 2 : 3); }
__host__ __device__ constexpr int lf(int f, int i) { return i < f ? i : i + 1; }

struct Species {
  int32_t ns;
  int64_t begin[kMaxSpecies + 1];
  double kq[kMaxSpecies];   // (q/m) dt / 2
  double qw[kMaxSpecies];   // q w
  float kq32[kMaxSpecies];  // kq rounded to FP32 (the mixed push's coefficient)
};

// Record of a particle that leaves its home tet: written by the common path
// into its tile's region of the crossing queue (contiguous, so the crossing
// kernel reads it coalesced instead of re-reading the SoA sparsely).
struct __align__(16) CrossRec {
  double a[3];
  float v[3];
  int32_t T;
  int32_t p;
};

// FP64-form record of a leaving particle: start point and new velocity in
// FP64.
struct __align__(16) CrossRec64 {
  double a[3];
  double v[3];
  int32_t T;
  int32_t p;
};

struct PushArgs {
  int64_t n;
  double* x;
  double* y;
  double* z;
  void* vx;
  void* vy;
  void* vz;
  int32_t* tet;
  uint8_t* status;
  int32_t* ncross;
  Species sp;
  double dt;
  float dt32;                   // dt rounded to FP32 (the mixed position update's step)
  int32_t max_cross;
  int32_t wall_mode;
  double lo[3], hi[3];
  int64_t nt, ne;
  const double* geom64;
  const float4* tetrec;
  const int4* tn;
  const int4* nb;
  const int4* te;
  const void* field;
  double* dG;                   // FP64 form accumulator [Ne]
  unsigned long long* dGq;      // 24-bit form: per (species, tet) slots of the 6 local edges,
                                // [ns][nt][8] int64 in units of 2^-48 (q w)
  double* mom;                  // contract form: per (species, tet) moment slots [ns][nt][6]:
                                // sum of D (3), sum of u x D (3), FP64
  float* momlo;                 // low FP32 parts of the crossing pass's moments [ns][nt][8]
  const float4* tetdf;          // contract form: low FP32 parts of grad lambda_1..3, [nt][4] float4
  unsigned long long* stats;    // [0] crossings, [1] frozen, [2] staging wait timeouts
  CrossRec* xrec;               // mixed form: crossing records, 256-slot region per tile
  CrossRec64* xrec64;           // FP64 form: the same, FP64 records
  int32_t* xcount;              // mixed form: records per tile
  unsigned long long wait_ns;   // limit of each bounded wait of the staged kernel
  int32_t stall_cta;            // test support: this CTA waits on a barrier nothing completes (-1: none)
};

__device__ __forceinline__ int species_of(const Species& sp, int64_t p) {
  int s = 0;
#pragma unroll 1
  while (s + 1 < sp.ns && p >= sp.begin[s + 1]) s++;
  return s;
}

// ------------------------------------------------------ debug bounds checks
// The library's debug build (compiled with FEMPIC_BOUNDS_CHECK) checks every
// index read from a mesh table against its range before it addresses
// memory: edge and face ids before a DoF load or a deposit, neighbour ids
// before the walk moves into the neighbour, node ids before a charge is
// assigned, adjacency slots before the edge pull reads them.  A bad index is
// counted in stats[3] (fempic_error_count then returns FEMPIC_EBOUNDS) and
// its access is skipped: a DoF reads as zero, a deposit term is dropped, a
// walking particle freezes with status LOST.  Nothing traps.  The release
// build compiles the checks out.
#ifdef FEMPIC_BOUNDS_CHECK
constexpr bool kBoundsCheck = true;
#else
constexpr bool kBoundsCheck = false;
#endif
__device__ __forceinline__ bool idx_in(int64_t i, int64_t n, unsigned long long* stats) {
  if (!kBoundsCheck) return true;
  if (i >= 0 && i < n) return true;
  if (stats) atomicAdd(stats + 3, 1ull);
  return false;
}

// ---------------------------------------------------------------- location
// Barycentrics with the fixed FP64 operation order (no contraction), so that
// point location reproduces exactly across implementations.
__device__ __forceinline__ void bary_exact(const double* __restrict__ g, double rx, double ry, double rz,
                                           double lam[4]) {
  const double dx = __dsub_rn(rx, g[0]), dy = __dsub_rn(ry, g[1]), dz = __dsub_rn(rz, g[2]);
#pragma unroll
  for (int k = 1; k < 4; k++) {
    const double* gk = g + 3 * k;
    lam[k] = __dadd_rn(__dadd_rn(__dmul_rn(gk[0], dx), __dmul_rn(gk[1], dy)), __dmul_rn(gk[2], dz));
  }
  lam[0] = __dsub_rn(__dsub_rn(__dsub_rn(1.0, lam[1]), lam[2]), lam[3]);
}

__device__ __forceinline__ int grid_cell_dev(double x, double lo, double ginv, int gd) {
  double f = floor(__dmul_rn(__dsub_rn(x, lo), ginv));
  if (!(f >= 0.0)) return 0;
  if (f > (double)(gd - 1)) return gd - 1;
  return (int)f;
}

struct LocateArgs {
  int64_t n;
  const double* x;
  const double* y;
  const double* z;
  int32_t* tet;
  uint8_t* status;
  const double* geom64;
  const int64_t* gstart;
  const int32_t* gtet;
  int gd[3];
  double ginv[3];
  double lo[3];
  int64_t nt;                 // bounds checks of the debug build
  unsigned long long* stats;
};

__global__ void __launch_bounds__(kThreads) k_locate(LocateArgs A) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= A.n) return;
  const double rx = A.x[p], ry = A.y[p], rz = A.z[p];
  int32_t found = -1;
  if (isfinite(rx) && isfinite(ry) && isfinite(rz)) {
    const int ci = grid_cell_dev(rx, A.lo[0], A.ginv[0], A.gd[0]);
    const int cj = grid_cell_dev(ry, A.lo[1], A.ginv[1], A.gd[1]);
    const int ck = grid_cell_dev(rz, A.lo[2], A.ginv[2], A.gd[2]);
    const int64_t c = ci + (int64_t)A.gd[0] * (cj + (int64_t)A.gd[1] * ck);
    const int64_t e = A.gstart[c + 1];
    for (int64_t i = A.gstart[c]; i < e; i++) {
      const int32_t t = A.gtet[i];
      if (!idx_in(t, A.nt, A.stats)) continue;
      double lam[4];
      bary_exact(A.geom64 + 12 * (int64_t)t, rx, ry, rz, lam);
      if (lam[0] >= 0.0 && lam[1] >= 0.0 && lam[2] >= 0.0 && lam[3] >= 0.0) {
        found = t;
        break;
      }
    }
  }
  A.tet[p] = found;
  A.status[p] = found < 0 ? FEMPIC_P_LOST : FEMPIC_P_OK;
}

// ------------------------------------------------------- field pre-pass
// Per tet: restore the carrier on the 10 DoFs (Re{c e~}), then express the
// Whitney expansion as an affine field about x0:
//   E(r) = E0 + d x W,  E0 = sum_j eps_0j g_j,  W = sum_{i<j} eps_ij (g_j x g_i)
//   B(r) = B0 + beta d, B0 = 2 (b1 g2 x g3 + b2 g1 x g3 + b3 g1 x g2),
//                       beta = 2 sum_f b_f det[g_f0, g_f1, g_f2]
// with d = r - x0 and g_0 = -(g_1 + g_2 + g_3).
template <typename R>
struct V3 {
  R x, y, z;
};
template <typename R>
__device__ __forceinline__ V3<R> vcross(V3<R> a, V3<R> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename R>
__device__ __forceinline__ R vdot(V3<R> a, V3<R> b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}

// Envelope DoF levels of one step and the carrier coefficient of each:
// level k enters as Re{c_k e^k} with c_k = a(t) e^{j omega0 t} N_k(t) (one
// level: N_0 = 1).
template <typename C2, typename R>
struct Levels {
  const C2* e[3];
  const C2* b[3];
  R cre[3], cim[3];
  int64_t ne, nf;                 // DoF counts (bounds checks of the debug build)
  unsigned long long* stats;
};

template <typename R, typename C2, int NL>
__device__ __forceinline__ void field_coeffs(const V3<R> g[4], const Levels<C2, R>& L, const int32_t* eid,
                                             const int32_t* fid, R out[10]) {
  R eps[6], bet[4];
#pragma unroll
  for (int e = 0; e < 6; e++) {
    R acc = 0;
    if (idx_in(eid[e], L.ne, L.stats)) {
      const C2 d = L.e[0][eid[e]];
      acc = L.cre[0] * d.x - L.cim[0] * d.y;
#pragma unroll
      for (int k = 1; k < NL; k++) {
        const C2 dk = L.e[k][eid[e]];
        acc += L.cre[k] * dk.x - L.cim[k] * dk.y;
      }
    }
    eps[e] = acc;
  }
#pragma unroll
  for (int f = 0; f < 4; f++) {
    R acc = 0;
    if (idx_in(fid[f], L.nf, L.stats)) {
      const C2 d = L.b[0][fid[f]];
      acc = L.cre[0] * d.x - L.cim[0] * d.y;
#pragma unroll
      for (int k = 1; k < NL; k++) {
        const C2 dk = L.b[k][fid[f]];
        acc += L.cre[k] * dk.x - L.cim[k] * dk.y;
      }
    }
    bet[f] = acc;
  }
  V3<R> E0 = {eps[0] * g[1].x + eps[1] * g[2].x + eps[2] * g[3].x,
              eps[0] * g[1].y + eps[1] * g[2].y + eps[2] * g[3].y,
              eps[0] * g[1].z + eps[1] * g[2].z + eps[2] * g[3].z};
  V3<R> W = {0, 0, 0};
#pragma unroll
  for (int e = 0; e < 6; e++) {
    const V3<R> c = vcross(g[le1(e)], g[le0(e)]);
    W.x += eps[e] * c.x;
    W.y += eps[e] * c.y;
    W.z += eps[e] * c.z;
  }
  const V3<R> c23 = vcross(g[2], g[3]), c13 = vcross(g[1], g[3]), c12 = vcross(g[1], g[2]);
  V3<R> B0 = {R(2) * (bet[1] * c23.x + bet[2] * c13.x + bet[3] * c12.x),
              R(2) * (bet[1] * c23.y + bet[2] * c13.y + bet[3] * c12.y),
              R(2) * (bet[1] * c23.z + bet[2] * c13.z + bet[3] * c12.z)};
  R beta = 0;
#pragma unroll
  for (int f = 0; f < 4; f++) {
    const V3<R> a = g[lf(f, 0)], b = g[lf(f, 1)], c = g[lf(f, 2)];
    beta += bet[f] * vdot(a, vcross(b, c));
  }
  beta *= R(2);
  out[0] = E0.x; out[1] = E0.y; out[2] = E0.z;
  out[3] = W.x;  out[4] = W.y;  out[5] = W.z;
  out[6] = B0.x; out[7] = B0.y; out[8] = B0.z;
  out[9] = beta;
}

template <int NL>
__global__ void __launch_bounds__(kThreads) k_field_fp64(int64_t nt, const double* __restrict__ geom64,
                                                          const int4* __restrict__ te, const int4* __restrict__ tf,
                                                          Levels<double2, double> L, double* __restrict__ field) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const double* G = geom64 + 12 * t;
  V3<double> g[4];
  g[1] = {G[3], G[4], G[5]};
  g[2] = {G[6], G[7], G[8]};
  g[3] = {G[9], G[10], G[11]};
  g[0] = {-(g[1].x + g[2].x + g[3].x), -(g[1].y + g[2].y + g[3].y), -(g[1].z + g[2].z + g[3].z)};
  const int4 e0 = te[2 * t], e1 = te[2 * t + 1], f = tf[t];
  const int32_t eid[6] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y};
  const int32_t fid[4] = {f.x, f.y, f.z, f.w};
  double out[10];
  field_coeffs<double, double2, NL>(g, L, eid, fid, out);
  double2* o = reinterpret_cast<double2*>(field + 10 * t);
#pragma unroll
  for (int i = 0; i < 5; i++) o[i] = make_double2(out[2 * i], out[2 * i + 1]);
}

template <int NL>
__global__ void __launch_bounds__(kThreads) k_field_f32(int64_t nt, float4* __restrict__ rec,
                                                         const int4* __restrict__ te, const int4* __restrict__ tf,
                                                         Levels<float2, float> L) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const float4 a = rec[8 * t + 1], b = rec[8 * t + 2], c = rec[8 * t + 3];
  V3<float> g[4];
  g[1] = {a.z, a.w, b.x};
  g[2] = {b.y, b.z, b.w};
  g[3] = {c.x, c.y, c.z};
  g[0] = {-(g[1].x + g[2].x + g[3].x), -(g[1].y + g[2].y + g[3].y), -(g[1].z + g[2].z + g[3].z)};
  const int4 e0 = te[2 * t], e1 = te[2 * t + 1], f = tf[t];
  const int32_t eid[6] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y};
  const int32_t fid[4] = {f.x, f.y, f.z, f.w};
  float out[10];
  field_coeffs<float, float2, NL>(g, L, eid, fid, out);
  rec[8 * t + 4] = make_float4(out[0], out[1], out[2], out[3]);
  rec[8 * t + 5] = make_float4(out[4], out[5], out[6], out[7]);
  reinterpret_cast<float2*>(rec + 8 * t + 6)[0] = make_float2(out[8], out[9]);   // z, w: face maps
}

// ------------------------------------------------------------ FP64 push
__device__ __forceinline__ void bary64_d(const double* __restrict__ g, double dx, double dy, double dz,
                                         double lam[4]) {
#pragma unroll
  for (int k = 1; k < 4; k++) {
    const double* gk = g + 3 * k;
    lam[k] = fma(gk[2], dz, fma(gk[1], dy, gk[0] * dx));
  }
  lam[0] = __dsub_rn(__dsub_rn(__dsub_rn(1.0, lam[1]), lam[2]), lam[3]);
}

__device__ __forceinline__ void bary64(const double* __restrict__ g, const double r[3], double lam[4]) {
  bary64_d(g, r[0] - g[0], r[1] - g[1], r[2] - g[2], lam);
}

// Sign and finiteness tests of doubles on their bit patterns: integer
// instructions instead of FP64 compares, which GB300 issues at the FP64 rate.
__device__ __forceinline__ bool finite_bits(double r) {
  return (((unsigned)__double2hiint(r) >> 20) & 0x7ffu) != 0x7ffu;
}

__device__ __forceinline__ bool negative_bits(double r) {   // r < 0 for finite r (-0 is not negative)
  const int hi = __double2hiint(r);
  return hi < 0 && (((unsigned)hi & 0x7fffffffu) | (unsigned)__double2loint(r)) != 0u;
}

__device__ __forceinline__ void deposit64(const PushArgs& A, int32_t T, const double la[4], const double lb[4],
                                          double qw) {
  if (!A.dG) return;   // deposits off
  const int4 e0 = __ldg(&A.te[2 * (int64_t)T]), e1 = __ldg(&A.te[2 * (int64_t)T + 1]);
  const int32_t eid[6] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y};
#pragma unroll
  for (int e = 0; e < 6; e++) {
    const int i = le0(e), j = le1(e);
    const double g = qw * fma(la[i], lb[j], -(la[j] * lb[i]));
    if (idx_in(eid[e], A.ne, A.stats)) atomicAdd(A.dG + eid[e], g);
  }
}

__device__ __forceinline__ int4 ldg_int4(const int4* p) { return __ldg(p); }

// FP64 form, common path: one particle per thread (a block is one 256-particle
// tile).  Gather, Boris, position update and the barycentrics of both ends
// in the home tet; a particle that stays deposits its segment and is done; a
// particle that leaves stores its new state provisionally and a record for
// the crossing pass, so the face walk does not run here with most lanes idle.
__global__ void __launch_bounds__(kThreads) k_push_fp64(PushArgs A) {
  __shared__ int32_t total;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  if (threadIdx.x == 0) total = 0;
  __syncthreads();
  unsigned nfrz = 0;
  bool leave = false;
  double a[3] = {0.0, 0.0, 0.0}, vn[3] = {0.0, 0.0, 0.0};
  int32_t T = -1;
  if (p < A.n) {
    T = A.tet[p];
    if (T >= A.nt) {
      A.tet[p] = -1;
      A.status[p] = FEMPIC_P_LOST;
      nfrz = 1;
    } else if (T >= 0) {
      const int s = species_of(A.sp, p);
      const double kq = A.sp.kq[s], qw = A.sp.qw[s];
      double* vxp = static_cast<double*>(A.vx);
      double* vyp = static_cast<double*>(A.vy);
      double* vzp = static_cast<double*>(A.vz);
      a[0] = A.x[p];
      a[1] = A.y[p];
      a[2] = A.z[p];
      const double v[3] = {vxp[p], vyp[p], vzp[p]};
      const double* G = A.geom64 + 12 * (int64_t)T;
      const double2* F = reinterpret_cast<const double2*>(static_cast<const double*>(A.field) + 10 * (int64_t)T);
      const double2 f0 = __ldg(F), f1 = __ldg(F + 1), f2 = __ldg(F + 2), f3 = __ldg(F + 3), f4 = __ldg(F + 4);
      const double dx = a[0] - __ldg(G), dy = a[1] - __ldg(G + 1), dz = a[2] - __ldg(G + 2);
      // (b)+(c) gather with the carrier already restored per tet
      const double Wx = f1.y, Wy = f2.x, Wz = f2.y;
      const double Ex = f0.x + (dy * Wz - dz * Wy);
      const double Ey = f0.y + (dz * Wx - dx * Wz);
      const double Ez = f1.x + (dx * Wy - dy * Wx);
      const double beta = f4.y;
      const double Bx = f3.x + beta * dx, By = f3.y + beta * dy, Bz = f4.x + beta * dz;
      // (d) Boris
      const double vmx = v[0] + kq * Ex, vmy = v[1] + kq * Ey, vmz = v[2] + kq * Ez;
      const double tx = kq * Bx, ty = kq * By, tz = kq * Bz;
      const double t2 = tx * tx + ty * ty + tz * tz;
      const double f = 2.0 / (1.0 + t2);
      const double sx = f * tx, sy = f * ty, sz = f * tz;
      const double vpx = vmx + (vmy * tz - vmz * ty);
      const double vpy = vmy + (vmz * tx - vmx * tz);
      const double vpz = vmz + (vmx * ty - vmy * tx);
      vn[0] = vmx + (vpy * sz - vpz * sy) + kq * Ex;
      vn[1] = vmy + (vpz * sx - vpx * sz) + kq * Ey;
      vn[2] = vmz + (vpx * sy - vpy * sx) + kq * Ez;
      const double b[3] = {fma(A.dt, vn[0], a[0]), fma(A.dt, vn[1], a[1]), fma(A.dt, vn[2], a[2])};
      if (!(finite_bits(vn[0]) && finite_bits(vn[1]) && finite_bits(vn[2]) && finite_bits(b[0]) &&
            finite_bits(b[1]) && finite_bits(b[2]))) {
        A.status[p] = FEMPIC_P_NONFINITE;
        A.tet[p] = -2 - T;
        nfrz = 1;
      } else {
        double la[4], lb[4];
        bary64_d(G, dx, dy, dz, la);
        bary64(G, b, lb);
        A.x[p] = b[0];
        A.y[p] = b[1];
        A.z[p] = b[2];
        vxp[p] = vn[0];
        vyp[p] = vn[1];
        vzp[p] = vn[2];
        leave = negative_bits(lb[0]) || negative_bits(lb[1]) || negative_bits(lb[2]) || negative_bits(lb[3]);
        if (!leave) deposit64(A, T, la, lb, qw);   // (f) the whole segment is in the home tet
      }
    }
  }
  // (e) leaving particles: records for the crossing pass, in the block's region
  const unsigned qmask = __ballot_sync(full, leave);
  if (qmask) {
    int base = 0;
    if (lane == 0) base = atomicAdd(&total, __popc(qmask));
    base = __shfl_sync(full, base, 0);
    if (leave) {
      CrossRec64& r = A.xrec64[blockIdx.x * (int64_t)kThreads + base + __popc(qmask & ((1u << lane) - 1u))];
      r.a[0] = a[0];
      r.a[1] = a[1];
      r.a[2] = a[2];
      r.v[0] = vn[0];
      r.v[1] = vn[1];
      r.v[2] = vn[2];
      r.T = T;
      r.p = (int32_t)p;
    }
  }
  nfrz = __reduce_add_sync(full, nfrz);
  if (lane == 0 && nfrz) atomicAdd(A.stats + 1, (unsigned long long)nfrz);
  __syncthreads();
  if (threadIdx.x == 0) A.xcount[blockIdx.x] = total;
}

// FP64 form, crossing pass: the walk of one leaving particle, one face per
// call, in FP64 (the paper's exit parameter s_k = la_k / (la_k - lb_k), the
// crossing point a + s (b - a), barycentrics carried exactly onto the
// neighbour's shared nodes).
struct CrossState64 {
  double a[3], b[3], vn[3];
  double la[4], lb[4];
  int32_t T, p;
  int entry, nc, s;
  uint8_t st;
  bool reflected;
};

__device__ __forceinline__ void cross64_begin(const PushArgs& A, const CrossRec64& r, CrossState64& c) {
  c.p = r.p;
  c.T = r.T;
  c.s = species_of(A.sp, r.p);
#pragma unroll
  for (int k = 0; k < 3; k++) {
    c.a[k] = r.a[k];
    c.vn[k] = r.v[k];
    c.b[k] = fma(A.dt, r.v[k], r.a[k]);
  }
  const double* G = A.geom64 + 12 * (int64_t)c.T;
  bary64(G, c.a, c.la);
  bary64(G, c.b, c.lb);
  c.entry = -1;
  c.nc = 0;
  c.st = FEMPIC_P_OK;
  c.reflected = false;
}

__device__ __forceinline__ bool cross64_advance(const PushArgs& A, CrossState64& c) {
  const double qw = A.sp.qw[c.s];
  int kx = -1;
  double smin = INFINITY;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    if (k == c.entry || !negative_bits(c.lb[k])) continue;
    double sk = c.la[k] / (c.la[k] - c.lb[k]);
    if (sk < 0.0) sk = 0.0;
    if (sk < smin) {
      smin = sk;
      kx = k;
    }
  }
  if (kx < 0) {
    deposit64(A, c.T, c.la, c.lb, qw);
#pragma unroll
    for (int k = 0; k < 3; k++) c.a[k] = c.b[k];
    return true;
  }
  double lp[4];
#pragma unroll
  for (int i = 0; i < 4; i++) lp[i] = (i == kx) ? 0.0 : fma(smin, c.lb[i] - c.la[i], c.la[i]);
  deposit64(A, c.T, c.la, lp, qw);
  c.nc++;
#pragma unroll
  for (int k = 0; k < 3; k++) c.a[k] = fma(smin, c.b[k] - c.a[k], c.a[k]);
  if (c.nc > A.max_cross) {
    c.st = FEMPIC_P_CAP;
    return true;
  }
  const int4 nbv = ldg_int4(&A.nb[c.T]);
  const int32_t nbt = kx == 0 ? nbv.x : kx == 1 ? nbv.y : kx == 2 ? nbv.z : nbv.w;
  if (nbt >= 0 && !idx_in(nbt, A.nt, A.stats)) {
    c.st = FEMPIC_P_LOST;
    return true;
  }
  if (nbt >= 0) {
    const int4 o4 = ldg_int4(&A.tn[c.T]), n4 = ldg_int4(&A.tn[nbt]);
    const int32_t on[4] = {o4.x, o4.y, o4.z, o4.w}, nn[4] = {n4.x, n4.y, n4.z, n4.w};
    int ent = 0;
#pragma unroll
    for (int i2 = 0; i2 < 4; i2++) {
      int hit = -1;
#pragma unroll
      for (int i = 0; i < 4; i++)
        if (on[i] == nn[i2]) hit = i;
      double val = 0.0;
#pragma unroll
      for (int i = 0; i < 4; i++)
        if (i == hit) val = lp[i];
      c.la[i2] = val;
      if (hit < 0) ent = i2;
    }
    c.T = nbt;
    c.entry = ent;
  } else if (nbt <= -1 && nbt >= -6 && A.wall_mode == FEMPIC_WALL_REFLECT) {
    const int code = -1 - nbt, ax = code >> 1, side = code & 1;
#pragma unroll
    for (int k = 0; k < 3; k++)
      if (k == ax) {
        const double L = side ? A.hi[k] : A.lo[k];
        c.b[k] = 2.0 * L - c.b[k];
        c.vn[k] = -c.vn[k];
      }
    c.reflected = true;
#pragma unroll
    for (int i = 0; i < 4; i++) c.la[i] = lp[i];
    c.entry = kx;
  } else {
    c.st = FEMPIC_P_ABSORBED;
    return true;
  }
  bary64(A.geom64 + 12 * (int64_t)c.T, c.b, c.lb);
  return false;
}

__device__ __forceinline__ void cross64_finish(const PushArgs& A, const CrossState64& c, unsigned& ncr,
                                               unsigned& nfrz) {
  const int64_t p = c.p;
  if (c.st != FEMPIC_P_OK || c.reflected) {   // otherwise a = b, already stored
    A.x[p] = c.a[0];
    A.y[p] = c.a[1];
    A.z[p] = c.a[2];
  }
  if (c.reflected) {
    static_cast<double*>(A.vx)[p] = c.vn[0];
    static_cast<double*>(A.vy)[p] = c.vn[1];
    static_cast<double*>(A.vz)[p] = c.vn[2];
  }
  int32_t T = c.T;
  if (c.st != FEMPIC_P_OK) {
    A.status[p] = c.st;
    T = -2 - T;
    nfrz++;
  }
  A.tet[p] = T;
  if (A.ncross) A.ncross[p] += c.nc;
  ncr += (unsigned)c.nc;
}

// One warp per group of tile regions (grid stride): the warp's tiles form one
// record stream, and lanes take the next record, across tile boundaries,
// when their particle is done.  The FP64 walk is FP64-pipe bound, so lanes
// left idle at the end of a tile would cost pipe cycles (the latency-bound
// mixed pass keeps the per-tile loop, which measured faster there).
__global__ void __launch_bounds__(kThreads) k_cross_fp64(PushArgs A, int64_t ntiles) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  unsigned ncr = 0, nfrz = 0;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  int64_t tile = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int32_t cnt = tile < ntiles ? A.xcount[tile] : 0, next = 0;
  bool have = false;
  CrossState64 c;
  for (;;) {
    unsigned idle = __ballot_sync(full, !have);
    while (idle && tile < ntiles) {   // warp-uniform: assigns records or advances a tile
      const int32_t avail = cnt - next;
      const int32_t want = __popc(idle);
      const int32_t take = avail < want ? avail : want;
      const int r = __popc(idle & lt);
      if (!have && r < take) {
        cross64_begin(A, A.xrec64[tile * kThreads + next + r], c);
        have = true;
      }
      next += take;
      idle = __ballot_sync(full, !have);
      if (next == cnt) {
        tile += warps;
        cnt = tile < ntiles ? A.xcount[tile] : 0;
        next = 0;
      }
    }
    if (!__any_sync(full, have)) break;
    if (have && cross64_advance(A, c)) {
      cross64_finish(A, c, ncr, nfrz);
      have = false;
    }
  }
  ncr = __reduce_add_sync(full, ncr);
  nfrz = __reduce_add_sync(full, nfrz);
  if (lane == 0) {
    if (ncr) atomicAdd(A.stats, (unsigned long long)ncr);
    if (nfrz) atomicAdd(A.stats + 1, (unsigned long long)nfrz);
  }
}

// ------------------------------------------------------------ mixed push
// Two FP32-mixed forms share the per-tet record, the gather, the carrier
// product and the Boris push in FP32 and keep positions in FP64:
//
//  * the contract form (FEMPIC_MIXED) keeps the quantities charge
//    conservation and tracking rest on at FP64 accuracy: r - x0 is one FP64
//    subtraction, the deposit of a particle that stays in its tet is the
//    exact moment form (below), and the face walk computes barycentrics,
//    exit parameters and crossing barycentrics in double-float (FP32 pairs,
//    a 48-bit significand) with the crossing point itself in FP64;
//  * the 24-bit form (FEMPIC_MIXED_Q24) fixes barycentrics to 24-bit integers
//    Q with Q_0 = 2^24 - Q_1 - Q_2 - Q_3, so sum(Q) = 2^24 exactly and the
//    per-segment deposit g_ij = Qa_i Qb_j - Qa_j Qb_i is exact in int64: its
//    edge divergence is exactly 2^24 (Qb - Qa) at the nodes, and charge is
//    conserved exactly at the resolution of the integers.
//
// GB300 issues FP64 at 1/64 of the FP32 rate, so the common path's only FP64
// arithmetic is r - x0 and the position update r + dt v.
//
// Mixed per-tet record tetrec (8 x float4 = 128 B):
//   bytes   0-23  x0 (node 0 of the tet) as 3 x f64, exact
//   bytes  24-59  grad lambda_1..3 in FP32 (9 floats)
//   bytes  60-63  kappa: error bound of the FP32 inside test (contract form)
//   bytes  64-103 the step's affine field (10 floats, k_field_f32)
//   bytes 104-111 four 16-bit face maps;  bytes 112-127 neighbour ids
struct FF {
  float hi, lo;
};

// Exact widening of a float to double with integer operations (rebias the
// exponent, shift the significand): GB300 runs the hardware conversion at
// the FP64 rate, 1/64 of the FP32 rate.  Zero keeps its sign; subnormal,
// infinite and NaN inputs take the hardware conversion, so the result is the
// double the conversion gives for every float.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu, sign = u & 0x80000000u;
  if (e - 1u >= 0xfeu) {
    if ((u << 1) == 0u) return __hiloint2double((int)sign, 0);
    return (double)f;
  }
  return __hiloint2double((int)(sign | ((e + 896u) << 20) | (m >> 3)), (int)(m << 29));
}

// r = hi + lo: hi keeps the leading 24 bits of the FP64 significand
// (truncated, so exactly a float), lo the remaining 29 bits rounded to FP32.
// |r| outside [2^-126, 2^128) maps to 0 (non-finite values are rejected
// before this is called).
__device__ __forceinline__ FF split_f64(double r) {
  const unsigned hi = (unsigned)__double2hiint(r), lo = (unsigned)__double2loint(r);
  const unsigned e = (hi >> 20) & 0x7ffu;
  if (e < 897u || e > 1150u) return FF{0.f, 0.f};
  const unsigned sign = hi & 0x80000000u;
  const float fhi = __uint_as_float(sign | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
  const float scale = e > 948u ? __uint_as_float((e - 948u) << 23) : 0.f;   // 2^(e - 1075)
  const float flo = __fmul_rn(__uint2float_rn(lo & 0x1fffffffu), scale);
  return FF{fhi, sign ? -flo : flo};
}

struct Geo32 {
  double x0[3];
  float g[9];    // grad lambda_1, _2, _3
  float kappa;
};

__device__ __forceinline__ Geo32 ld_geo(const float4* __restrict__ rec, int64_t T) {
  const float4 a = __ldg(rec + 8 * T), b = __ldg(rec + 8 * T + 1), c = __ldg(rec + 8 * T + 2),
               d = __ldg(rec + 8 * T + 3);
  Geo32 G;
  G.x0[0] = __hiloint2double(__float_as_int(a.y), __float_as_int(a.x));
  G.x0[1] = __hiloint2double(__float_as_int(a.w), __float_as_int(a.z));
  G.x0[2] = __hiloint2double(__float_as_int(b.y), __float_as_int(b.x));
  G.g[0] = b.z; G.g[1] = b.w; G.g[2] = c.x;
  G.g[3] = c.y; G.g[4] = c.z; G.g[5] = c.w;
  G.g[6] = d.x; G.g[7] = d.y; G.g[8] = d.z;
  G.kappa = d.w;
  return G;
}

// d = r - x0: one FP64 subtraction (exact for points in or near the tet,
// whose coordinates are close to x0's), split into an FP32 pair d = hi + lo
// (lo keeps d to 2^-48 relative), and rounded to FP32 in d32.
__device__ __forceinline__ void dpos(const Geo32& G, double rx, double ry, double rz, FF dd[3], float d32[3]) {
  dd[0] = split_f64(__dsub_rn(rx, G.x0[0]));
  dd[1] = split_f64(__dsub_rn(ry, G.x0[1]));
  dd[2] = split_f64(__dsub_rn(rz, G.x0[2]));
#pragma unroll
  for (int k = 0; k < 3; k++) d32[k] = __fadd_rn(dd[k].hi, dd[k].lo);
}

__device__ __forceinline__ void bary_q(const Geo32& G, const float d[3], int32_t Q[4]) {
  const float l1 = __fmaf_rn(G.g[2], d[2], __fmaf_rn(G.g[1], d[1], __fmul_rn(G.g[0], d[0])));
  const float l2 = __fmaf_rn(G.g[5], d[2], __fmaf_rn(G.g[4], d[1], __fmul_rn(G.g[3], d[0])));
  const float l3 = __fmaf_rn(G.g[8], d[2], __fmaf_rn(G.g[7], d[1], __fmul_rn(G.g[6], d[0])));
  // |lambda| <= 32 keeps Q_0 = 2^24 - Q_1 - Q_2 - Q_3 inside int32 for points
  // up to 32 tet diameters away (a clamped point still tracks cell by cell).
  Q[1] = __float2int_rn(__fmul_rn(fminf(fmaxf(l1, -kQClamp), kQClamp), kQScale));
  Q[2] = __float2int_rn(__fmul_rn(fminf(fmaxf(l2, -kQClamp), kQClamp), kQScale));
  Q[3] = __float2int_rn(__fmul_rn(fminf(fmaxf(l3, -kQClamp), kQClamp), kQScale));
  Q[0] = kQOne - Q[1] - Q[2] - Q[3];
}

// Barycentric integers of the FP64 point r in tet T (shared with the nodal
// charge so that the charge assignment is the very function the deposit uses).
__device__ __forceinline__ void bary_q_at(const float4* __restrict__ geo, int64_t T, const double r[3],
                                          int32_t Q[4]) {
  const Geo32 G = ld_geo(geo, T);
  FF dd[3];
  float d[3];
  dpos(G, r[0], r[1], r[2], dd, d);
  bary_q(G, d, Q);
}

__device__ __forceinline__ void gq(const int32_t a[4], const int32_t b[4], long long g[6]) {
#pragma unroll
  for (int e = 0; e < 6; e++) {
    const int i = le0(e), j = le1(e);
    g[e] = (long long)a[i] * b[j] - (long long)a[j] * b[i];
  }
}

// The mixed form deposits into one 64-byte slot per (species, tet): the 6
// local edges of the tet, contiguous, so a run head touches 2 sectors instead
// of 6 scattered edge entries; k_deposit_finalize pulls each edge's sum from
// the slots of its incident tets.
__device__ __forceinline__ unsigned long long* tet_slot(const PushArgs& A, int s, int32_t T) {
  return A.dGq + ((int64_t)s * A.nt + T) * 8;
}

__device__ __forceinline__ void depositq_atomic(const PushArgs& A, int32_t T, int s, const long long g[6]) {
  if (!A.dGq) return;   // deposits off
  unsigned long long* base = tet_slot(A, s, T);
#pragma unroll
  for (int e = 0; e < 6; e++)
    if (g[e]) atomicAdd(base + e, (unsigned long long)g[e]);
}

// Exit face of the straight piece with end barycentrics Qa -> Qb in one tet,
// the entry face excluded: among faces with Qb_k < 0, the one whose crossing
// parameter s_k = Qa_k / (Qa_k - Qb_k) (clamped at 0) is smallest, the lowest
// k on ties; -1 when the piece stays inside.
__device__ __forceinline__ int exit_face(const int32_t Qa[4], const int32_t Qb[4], int entry, float& smin) {
  int kx = -1;
  smin = INFINITY;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    if (k == entry || Qb[k] >= 0) continue;
    const int32_t den = Qa[k] - Qb[k];
    float sk = den > 0 ? (float)Qa[k] / (float)den : 0.0f;
    if (sk < 0.0f) sk = 0.0f;
    if (sk < smin) {
      smin = sk;
      kx = k;
    }
  }
  return kx;
}

// Barycentric integers of the crossing point Qa + s (Qb - Qa) on exit face
// kx: exactly zero on that face, the sum kept at 2^24 on the last other node.
__device__ __forceinline__ void crossing_q(const int32_t Qa[4], const int32_t Qb[4], int kx, float smin,
                                           int32_t Qp[4]) {
  const int last = kx == 3 ? 2 : 3;
  int32_t acc = 0;
#pragma unroll
  for (int j = 0; j < 4; j++) {
    if (j == kx) {
      Qp[j] = 0;
    } else {
      Qp[j] = Qa[j] + __float2int_rn(smin * (float)(Qb[j] - Qa[j]));
      acc += Qp[j];
    }
  }
#pragma unroll
  for (int j = 0; j < 4; j++)
    if (j == last) Qp[j] += kQOne - acc;
}

// Position after the push: the one FP64 addition per coordinate of the
// common path.  Every mixed kernel forms it with this exact sequence, so the
// crossing kernels rebuild b from the stored start point and velocity bit
// for bit.
__device__ __forceinline__ double advance(double a, float dt32, float v) {
  return __dadd_rn(a, f32_to_f64(__fmul_rn(dt32, v)));
}

// ------------------------------------------------- double-float arithmetic
// A value h + l held as an FP32 pair (|l| below an ulp of h): a 48-bit
// significand at FP32 speed.  Built on the error-free transformations of
// Knuth (two-sum), Dekker (fast two-sum, |a| >= |b|) and the fused
// multiply-add product; the _rn intrinsics keep the compiler from
// contracting or reassociating the error terms away.
struct DF {
  float h, l;
};

__device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return DF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return DF{p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const DF s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.h, -a.l}; }
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const DF p = two_prod(a.h, b.h);
  return fast_two_sum(p.h, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l)));
}
__device__ __forceinline__ DF df_div(DF a, DF b) {
  const float q1 = __fdiv_rn(a.h, b.h);
  const DF p = two_prod(q1, b.h);
  // remainder a - q1 b, to first order in the low parts
  const float r = __fsub_rn(__fadd_rn(__fsub_rn(__fsub_rn(a.h, p.h), p.l), a.l), __fmul_rn(q1, b.l));
  return fast_two_sum(q1, __fdiv_rn(r, b.h));
}
__device__ __forceinline__ bool df_lt(DF a, DF b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
__device__ __forceinline__ DF df_dot3(const DF a[3], const DF b[3]) {
  return df_add(df_add(df_mul(a[0], b[0]), df_mul(a[1], b[1])), df_mul(a[2], b[2]));
}
// FP64 value of h + l; the FP64 addition is exact (the pair spans at most
// 48 bits).
__device__ __forceinline__ double df_to_f64(DF a) { return __dadd_rn(f32_to_f64(a.h), f32_to_f64(a.l)); }
__device__ __forceinline__ DF f64_to_df(double r) {
  const FF s = split_f64(r);
  return DF{s.hi, s.lo};
}

// ------------------------------------------------- contract-form deposit
// Moment form of the exact path integral of a straight segment a -> b that
// stays in one tet (Sec. III-D eq. G_integral with the Whitney-1 functions
// of Sec. III-A).  With u = a - x0 and D = b - a, lambda is affine, so
//   g_ij = lambda_i(a) lambda_j(b) - lambda_j(a) lambda_i(b)
//        = [i = 0] (G_j . D) + (G_i x G_j) . (u x D)      (G_k = grad lambda_k)
// (Binet-Cauchy).  Per particle only D and the moment u x D are needed, in
// physical units: D is exactly the FP32 displacement dt v of the mixed
// position update, u is exact from the FP64 subtraction, and u x D is
// formed as an FP32 pair from exact products.  The gradients enter once per
// tet per step, in double-float, in k_tet_finalize: FP64 accuracy without
// FP64 arithmetic per particle.
//
// Warp reduction: the 6 values of each lane (D and u x D) are scaled to
// integers by a quantum common to the warp (2^-50 of the warp's largest
// |D|, resp. |u x D|), summed exactly over runs of equal (tet, species)
// like the 24-bit form's integers, and the run head adds the sums, as FP64,
// to the tet's moment slot with FP64 atomics.

// Per-warp fixed point, as two 32-bit limbs: with y = x s (s a power of two,
// so the product is exact) the integer X = round(y 2^25) is held as hi 2^25
// + lo, hi = floor(y) and lo = round((y - hi) 2^25) in [0, 2^25].  With |y| <
// 2^25 for the warp's largest |x| (fx_scale), |X| < 2^50, and the sums of a
// warp's limbs stay below 2^31 in magnitude.  Float operations only: the
// floor and the two 32-bit conversions.
__device__ __forceinline__ void fx_limbs(float x, float scale, int& hi, unsigned& lo) {
  const float y = __fmul_rn(x, scale);
  const float h = floorf(y);
  hi = __float2int_rn(h);
  lo = __float2uint_rn(__fmul_rn(__fsub_rn(y, h), 33554432.0f));   // exact before the rounding
}

// s = 2^(151 - emax) for a warp whose largest |x| has biased exponent emax
// (|x| < 2^(emax - 126)), so |y| < 2^25 and X = x 2^(176 - emax).  0 when
// emax < 24 (every |x| below 2^-103, the values are dropped).
__device__ __forceinline__ float fx_scale(unsigned emax) {
  return emax < 24u ? 0.f : __uint_as_float((278u - emax) << 23);
}

__device__ __forceinline__ unsigned abs_bits(float x) { return __float_as_uint(x) & 0x7fffffffu; }

// Per-lane result of the common path, consumed by the warp epilogue.
struct LaneOut {
  long long gh[6];     // 24-bit form: one-segment deposit (home tet), int64
  float mv[9];         // contract form: D (3), u x D as pairs (hi 3, lo 3)
  int lh[6];           // the six values as 32-bit limbs (hi 2^25 + lo), for the run sums
  unsigned ll[6];
  int32_t key;         // (home tet, species) run key; negative = no deposit
  int32_t Thome;
  int shome;
  bool queue;          // leaves its tet (or may): tracked by the crossing pass
  unsigned nfrz;
  double a[3];         // start point and new velocity of a queued particle
  float v[3];
  int32_t T;
};

struct CrossList {
  int32_t total;     // records of the current tile
  long long sums[kThreads / 32][32 * 6];   // per warp: run sums of the deposit, by head lane
  int32_t keys[kThreads / 32][32];         // per warp: run keys, by head lane
};

__device__ __forceinline__ void lane_init(LaneOut& o, int lane) {
#pragma unroll
  for (int e = 0; e < 6; e++) o.gh[e] = 0;
#pragma unroll
  for (int e = 0; e < 9; e++) o.mv[e] = 0.f;
  o.key = -1 - lane;
  o.Thome = 0;
  o.shome = 0;
  o.queue = false;
  o.nfrz = 0;
}

// Common path of one particle with its state already loaded: gather, carrier,
// Boris, position update, then the inside test of the end point in the home
// tet.  A particle that stays in its tet writes its new state and keeps its
// one-segment deposit for the warp reduction; any other hands (start point,
// velocity, tet) to the CTA's crossing list.
//   24-bit form: inside = all four integer barycentrics of b >= 0.
//   contract form: inside = all four FP32 barycentrics of b >= kappa, the
//   tet's bound on their error, so that the FP64 barycentrics are >= 0 too;
//   a particle within kappa of a face goes to the crossing pass, which
//   decides in double-float.
template <bool Q24>
__device__ __forceinline__ void mixed_particle(const PushArgs& A, int64_t p, int32_t T, double ax, double ay,
                                               double az, float v0, float v1, float v2, LaneOut& o) {
  if (T >= A.nt) {
    A.tet[p] = -1;
    A.status[p] = FEMPIC_P_LOST;
    o.nfrz = 1;
    return;
  }
  if (T < 0) return;
  const int s = species_of(A.sp, p);
  const float kq = A.sp.kq32[s];
  const float4* R = A.tetrec + 8 * (int64_t)T;
  const Geo32 G = ld_geo(A.tetrec, T);
  const float4 f0 = __ldg(R + 4), f1 = __ldg(R + 5), f2 = __ldg(R + 6);
  FF dd[3];
  float d[3];
  dpos(G, ax, ay, az, dd, d);
  // f0 = (E0x, E0y, E0z, Wx), f1 = (Wy, Wz, B0x, B0y), f2 = (B0z, beta, -, -)
  const float Ex = f0.x + (d[1] * f1.y - d[2] * f1.x);
  const float Ey = f0.y + (d[2] * f0.w - d[0] * f1.y);
  const float Ez = f0.z + (d[0] * f1.x - d[1] * f0.w);
  const float Bx = f1.z + f2.y * d[0], By = f1.w + f2.y * d[1], Bz = f2.x + f2.y * d[2];
  const float vmx = v0 + kq * Ex, vmy = v1 + kq * Ey, vmz = v2 + kq * Ez;
  const float tx = kq * Bx, ty = kq * By, tz = kq * Bz;
  const float t2 = tx * tx + ty * ty + tz * tz;
  const float f = 2.0f / (1.0f + t2);
  const float sx = f * tx, sy = f * ty, sz = f * tz;
  const float vpx = vmx + (vmy * tz - vmz * ty);
  const float vpy = vmy + (vmz * tx - vmx * tz);
  const float vpz = vmz + (vmx * ty - vmy * tx);
  const float vn0 = vmx + (vpy * sz - vpz * sy) + kq * Ex;
  const float vn1 = vmy + (vpz * sx - vpx * sz) + kq * Ey;
  const float vn2 = vmz + (vpx * sy - vpy * sx) + kq * Ez;
  const float dt32 = A.dt32;
  // the FP32 displacement and the FP64 position update (advance's sequence)
  const float D0 = __fmul_rn(dt32, vn0), D1 = __fmul_rn(dt32, vn1), D2 = __fmul_rn(dt32, vn2);
  const double b0 = __dadd_rn(ax, f32_to_f64(D0)), b1 = __dadd_rn(ay, f32_to_f64(D1)),
               b2 = __dadd_rn(az, f32_to_f64(D2));
  if (!(isfinite(vn0) && isfinite(vn1) && isfinite(vn2) && finite_bits(b0) && finite_bits(b1) && finite_bits(b2))) {
    A.status[p] = FEMPIC_P_NONFINITE;
    A.tet[p] = -2 - T;
    o.nfrz = 1;
    return;
  }
  int32_t Qa[4], Qb[4];
  bool inside;
  if (Q24) {
    bary_q(G, d, Qa);
    FF bd[3];
    float db[3];
    dpos(G, b0, b1, b2, bd, db);
    bary_q(G, db, Qb);
    inside = (Qb[0] | Qb[1] | Qb[2] | Qb[3]) >= 0;
  } else {
    const float e0 = __fadd_rn(d[0], D0), e1 = __fadd_rn(d[1], D1), e2 = __fadd_rn(d[2], D2);
    const float l1 = __fmaf_rn(G.g[2], e2, __fmaf_rn(G.g[1], e1, __fmul_rn(G.g[0], e0)));
    const float l2 = __fmaf_rn(G.g[5], e2, __fmaf_rn(G.g[4], e1, __fmul_rn(G.g[3], e0)));
    const float l3 = __fmaf_rn(G.g[8], e2, __fmaf_rn(G.g[7], e1, __fmul_rn(G.g[6], e0)));
    const float l0 = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, l1), l2), l3);
    inside = fminf(fminf(l0, l1), fminf(l2, l3)) >= G.kappa;
  }
  // Every lane stores its full new state, a queued particle included (its b
  // is final unless it reflects or freezes), so the warp's stores cover whole
  // sectors and the crossing kernel rarely rewrites positions.
  static_cast<float*>(A.vx)[p] = vn0;
  static_cast<float*>(A.vy)[p] = vn1;
  static_cast<float*>(A.vz)[p] = vn2;
  A.x[p] = b0;
  A.y[p] = b1;
  A.z[p] = b2;
  if (!inside) {
    // the crossing pass deposits all its pieces (doing the home piece here
    // instead measured slower: the divergent exit search costs the common
    // path more than the crossing pass saves)
    o.queue = true;
    o.a[0] = ax;
    o.a[1] = ay;
    o.a[2] = az;
    o.v[0] = vn0;
    o.v[1] = vn1;
    o.v[2] = vn2;
    o.T = T;
    // joins its tet's run with zero values, so that the run is not split
    o.key = T * kMaxSpecies + s;
    return;
  }
  if (Q24) {
    gq(Qa, Qb, o.gh);
  } else {
    // u x D as FP32 pairs: exact products of the high parts, first-order low parts
    const float D[3] = {D0, D1, D2};
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const int i = (k + 1) % 3, j = (k + 2) % 3;   // (u x D)_k = u_i D_j - u_j D_i
      const DF p1 = two_prod(dd[i].hi, D[j]), p2 = two_prod(dd[j].hi, D[i]);
      const DF sd = two_sum(p1.h, -p2.h);
      o.mv[3 + k] = sd.h;
      o.mv[6 + k] = __fmaf_rn(dd[i].lo, D[j], __fmaf_rn(-dd[j].lo, D[i], __fadd_rn(sd.l, __fsub_rn(p1.l, p2.l))));
      o.mv[k] = D[k];
    }
  }
  o.key = T * kMaxSpecies + s;
  o.Thome = T;
  o.shome = s;
}

// Warp epilogue (all 32 lanes): append the queued lanes to the CTA's
// crossing list (one shared-memory atomic per warp), reduce the one-segment
// deposits over runs of equal (tet, species) keys (particles are sorted by
// tet, so neighbouring lanes usually share one), and flush them from the run
// head: int64 atomics into the tet's integer slot (24-bit form), or FP64
// atomics of the exactly summed moments into the tet's moment slot
// (contract form).
template <bool Q24>
__device__ __forceinline__ void mixed_warp_epilogue(const PushArgs& A, int64_t p, int lane, LaneOut& o,
                                                    CrossList& cl) {
  const unsigned full = 0xffffffffu;
  const unsigned qmask = __ballot_sync(full, o.queue);
  if (qmask) {
    int base = 0;
    if (lane == 0) base = atomicAdd(&cl.total, __popc(qmask));
    base = __shfl_sync(full, base, 0);
    if (o.queue) {
      CrossRec& r = A.xrec[(p & ~(int64_t)(kThreads - 1)) + base + __popc(qmask & ((1u << lane) - 1u))];
      r.a[0] = o.a[0];
      r.a[1] = o.a[1];
      r.a[2] = o.a[2];
      r.v[0] = o.v[0];
      r.v[1] = o.v[1];
      r.v[2] = o.v[2];
      r.T = o.T;
      r.p = (int32_t)p;
    }
  }
  const bool dep_on = Q24 ? (A.dGq != nullptr) : (A.mom != nullptr);
  if (dep_on) {   // deposits on (kernel parameter: the same branch for every lane)
    unsigned eD = 0u, eM = 0u;
    if (!Q24) {
      // the warp's quanta, then every lane's values as limbs
      unsigned uD = 0u, uM = 0u;
      if (o.key >= 0) {
        uD = max(max(abs_bits(o.mv[0]), abs_bits(o.mv[1])), abs_bits(o.mv[2]));
        uM = max(max(abs_bits(o.mv[3]), abs_bits(o.mv[4])), abs_bits(o.mv[5]));
      }
      eD = __reduce_max_sync(full, uD) >> 23;
      eM = __reduce_max_sync(full, uM) >> 23;
      const float sD = fx_scale(eD), sM = fx_scale(eM);
#pragma unroll
      for (int k = 0; k < 3; k++) {
        fx_limbs(o.mv[k], sD, o.lh[k], o.ll[k]);
        int h2;
        unsigned l2;
        fx_limbs(o.mv[3 + k], sM, o.lh[3 + k], o.ll[3 + k]);
        fx_limbs(o.mv[6 + k], sM, h2, l2);
        o.lh[3 + k] += h2;
        o.ll[3 + k] += l2;
      }
    }
    // exact sums over runs of equal (tet, species) keys (particles are sorted
    // by tet, so neighbouring lanes usually share one): a segmented
    // shuffle-down scan, as many rounds as the warp's longest run needs,
    // leaves each run's sums in its head lane
    const int32_t prev = __shfl_up_sync(full, o.key, 1);
    const bool head = lane == 0 || prev != o.key;
    const unsigned heads = __ballot_sync(full, head);
    const unsigned above = lane == 31 ? 0u : (heads & (~0u << (lane + 1)));
    const int run_end = above ? (__ffs(above) - 2) : 31;
    const unsigned longest = __reduce_max_sync(full, head ? (unsigned)(run_end - lane + 1) : 0u);
#pragma unroll 1
    for (int off = 1; off < (int)longest; off <<= 1) {
      const bool in = lane + off <= run_end;
#pragma unroll
      for (int e = 0; e < 6; e++) {
        if (Q24) {
          const long long v = __shfl_down_sync(full, o.gh[e], off);
          if (in) o.gh[e] += v;
        } else {
          const int vh = __shfl_down_sync(full, o.lh[e], off);
          const unsigned vl = __shfl_down_sync(full, o.ll[e], off);
          if (in) {
            o.lh[e] += vh;
            o.ll[e] += vl;
          }
        }
      }
    }
    // the slot updates: each head leaves its run's sums and key in the warp's
    // scratch rows, and the warp's (run, component) pairs are spread over its
    // lanes, 32 per round (one round for up to 5 runs)
    const int w = threadIdx.x >> 5;
    long long* row = cl.sums[w];
    const bool dep = o.key >= 0;
    if (head && dep) {
#pragma unroll
      for (int e = 0; e < 6; e++)
        row[6 * lane + e] = Q24 ? o.gh[e] : (long long)o.lh[e] * 33554432ll + (long long)o.ll[e];
      cl.keys[w][lane] = o.key;
    }
    const unsigned dheads = heads & __ballot_sync(full, dep);
    __syncwarp();
    const int npairs = 6 * __popc(dheads);
#pragma unroll 1
    for (int j = lane; j < npairs; j += 32) {
      const int r = j / 6, c = j - 6 * r;
      const int start = (int)__fns(dheads, 0, r + 1);
      const long long v = row[6 * start + c];
      if (v == 0) continue;
      const int32_t key = cl.keys[w][start];
      const int64_t slot = (int64_t)(key & (kMaxSpecies - 1)) * A.nt + (key / kMaxSpecies);
      if (Q24)
        atomicAdd(A.dGq + slot * 8 + c, (unsigned long long)v);
      else   // the run's X sum times 2^(emax - 176)
        atomicAdd(A.mom + slot * 6 + c,   // the hardware conversion: a few lanes per run, the FP64 pipe has room
                  (double)v * __longlong_as_double((long long)((int)(c < 3 ? eD : eM) - 176 + 1023) << 52));
    }
    __syncwarp();
  }
  const unsigned nf = __reduce_add_sync(full, o.nfrz);
  if (lane == 0 && nf) atomicAdd(A.stats + 1, (unsigned long long)nf);
}

// End of a tile (all threads, after the tile's epilogues): publish the tile's
// record count for the crossing kernel and reset the counter.
__device__ __forceinline__ void publish_tile(const PushArgs& A, CrossList& cl, int64_t tile) {
  __syncthreads();
  if (threadIdx.x == 0) {
    A.xcount[tile] = cl.total;
    cl.total = 0;
  }
}

// Common path, one particle per thread, state read straight from global
// memory.  Used when the particle arrays are not 16-byte aligned (so bulk
// copies cannot stage them) and for a ragged last tile.
template <bool Q24>
__global__ void __launch_bounds__(kThreads) k_push_mixed(PushArgs A, int64_t p0) {
  __shared__ CrossList cl;
  const int64_t p = p0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) cl.total = 0;
  __syncthreads();
  LaneOut o;
  lane_init(o, lane);
  if (p < A.n) {
    const int32_t T = A.tet[p];
    if (T >= 0) {
      const float* vx = static_cast<const float*>(A.vx);
      const float* vy = static_cast<const float*>(A.vy);
      const float* vz = static_cast<const float*>(A.vz);
      mixed_particle<Q24>(A, p, T, A.x[p], A.y[p], A.z[p], vx[p], vy[p], vz[p], o);
    } else {
      mixed_particle<Q24>(A, p, T, 0.0, 0.0, 0.0, 0.f, 0.f, 0.f, o);
    }
  }
  mixed_warp_epilogue<Q24>(A, p, lane, o, cl);
  publish_tile(A, cl, (p0 >> 8) + blockIdx.x);
}

// ------------------------------------------------- staged common path (TMA)
// Persistent CTAs walk full 256-particle tiles.  Each tile's slices of the
// seven particle arrays (x, y, z f64; vx, vy, vz f32; tet i32; 10 KB) are
// brought into shared memory by cp.async.bulk copies completing on an
// mbarrier, in a ring of three stages filled two tiles ahead, so HBM latency
// overlaps the arithmetic.  A stage is refilled only after the iteration
// that read it has finished on every thread.
// Every wait is bounded by the global timer (about 1 s by default); a CTA
// that times out records it in stats[2], drains the copies it issued, and
// stops.
constexpr int kTile = kThreads;
constexpr int kStageBytes = kTile * (3 * 8 + 3 * 4 + 4);   // 10240
constexpr int kStages = 3;
constexpr unsigned long long kWaitLimitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of `bar`; false after limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_test(bar, parity)) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}

__device__ __forceinline__ void stage_tile(const PushArgs& A, unsigned char* stage, int64_t tile, uint64_t* bar) {
  const int64_t p0 = tile * kTile;
  mbar_expect_tx(bar, kStageBytes);
  bulk_g2s(stage, A.x + p0, kTile * 8, bar);
  bulk_g2s(stage + kTile * 8, A.y + p0, kTile * 8, bar);
  bulk_g2s(stage + kTile * 16, A.z + p0, kTile * 8, bar);
  bulk_g2s(stage + kTile * 24, static_cast<const float*>(A.vx) + p0, kTile * 4, bar);
  bulk_g2s(stage + kTile * 28, static_cast<const float*>(A.vy) + p0, kTile * 4, bar);
  bulk_g2s(stage + kTile * 32, static_cast<const float*>(A.vz) + p0, kTile * 4, bar);
  bulk_g2s(stage + kTile * 36, A.tet + p0, kTile * 4, bar);
}

#ifndef FEMPIC_USE_TMA
#define FEMPIC_USE_TMA 1
#endif
#ifndef FEMPIC_TMA_MIN_BLOCKS
#define FEMPIC_TMA_MIN_BLOCKS 4
#endif
template <bool Q24>
__global__ void __launch_bounds__(kThreads, FEMPIC_TMA_MIN_BLOCKS) k_push_mixed_tma(PushArgs A, int64_t ntiles) {
  __shared__ __align__(128) unsigned char smem[kStages][kStageBytes];
  // bar[kStages] is test support: a barrier no copy ever completes, for the
  // CTA that fempic_debug_stall names
  __shared__ __align__(8) uint64_t bar[kStages + 1];
  __shared__ CrossList cl;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
    for (int k = 0; k <= kStages; k++) mbar_init(&bar[k], 1);
    mbar_fence_init();
    cl.total = 0;
  }
  __syncthreads();
  const int64_t stride = gridDim.x;
  const int64_t t0 = blockIdx.x;
  if (tid == 0)
    for (int k = 0; k < kStages; k++)
      if (t0 + k * stride < ntiles) stage_tile(A, smem[k], t0 + k * stride, &bar[k]);
  uint32_t phase = 0u;   // bit k = parity of the next wait on stage k
  int st = 0;
  for (int64_t it = 0, tile = t0; tile < ntiles; tile += stride, it++) {
    // Every thread finished iteration it-1 (which used stage st-1) before
    // this barrier; the proxy fence orders those shared-memory reads before
    // the bulk copy that refills that stage below.
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    bool ok = mbar_wait_bounded(&bar[st], (phase >> st) & 1u, A.wait_ns);
    if (it == 0 && (int)blockIdx.x == A.stall_cta) ok = ok && mbar_wait_bounded(&bar[kStages], 0u, A.wait_ns);
    if (__syncthreads_or(!ok)) {
      // give up: record it, wait (bounded) for this CTA's copies still in
      // flight (stages of tiles it .. it+kStages-1 not yet consumed), stop
      if (tid == 0) {
        atomicAdd(A.stats + 2, 1ull);
        for (int64_t t = tile; t < ntiles; t += stride) A.xcount[t] = 0;   // no stale records
        for (int k = 0; k < kStages; k++) {
          const int sk = (st + k) % kStages;
          if (tile + k * stride < ntiles) mbar_wait_bounded(&bar[sk], (phase >> sk) & 1u, A.wait_ns);
        }
      }
      return;
    }
    phase ^= 1u << st;
    if (tid == 0 && it > 0) {
      const int prev = (st + kStages - 1) % kStages;
      const int64_t next = tile + (kStages - 1) * stride;
      if (next < ntiles) stage_tile(A, smem[prev], next, &bar[prev]);
    }
    const unsigned char* S = smem[st];
    const double ax = reinterpret_cast<const double*>(S)[tid];
    const double ay = reinterpret_cast<const double*>(S + kTile * 8)[tid];
    const double az = reinterpret_cast<const double*>(S + kTile * 16)[tid];
    const float v0 = reinterpret_cast<const float*>(S + kTile * 24)[tid];
    const float v1 = reinterpret_cast<const float*>(S + kTile * 28)[tid];
    const float v2 = reinterpret_cast<const float*>(S + kTile * 32)[tid];
    const int32_t T = reinterpret_cast<const int32_t*>(S + kTile * 36)[tid];
    const int64_t p = tile * kTile + tid;
    LaneOut o;
    lane_init(o, lane);
    mixed_particle<Q24>(A, p, T, ax, ay, az, v0, v1, v2, o);
    mixed_warp_epilogue<Q24>(A, p, lane, o, cl);
    publish_tile(A, cl, tile);
    st = (st + 1) % kStages;
  }
}

// Crossing path of a particle that leaves its home tet, one face at a time.
// State of the walk: the current straight piece runs from a0 + sacc (b - a0)
// to b inside tet T, with end barycentrics Qa -> Qb; `entry` is the face it
// came in through.
struct CrossState {
  double a0[3], b[3];
  float vn[3];
  int32_t Qa[4], Qb[4];
  int32_t T, p;
  int entry, nc, s;
  float sacc;
  uint8_t st;
  bool moved, reflected;
};

// Start from the record: rebuild b bit for bit (the common path's sequence).
// The barycentrics follow in the first step (cross_advance with fresh).
__device__ __forceinline__ void cross_begin(const PushArgs& A, const CrossRec& r, CrossState& c) {
  c.p = r.p;
  c.T = r.T;
  c.s = species_of(A.sp, r.p);
  const float dt32 = A.dt32;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    c.a0[k] = r.a[k];
    c.vn[k] = r.v[k];
    c.b[k] = advance(r.a[k], dt32, r.v[k]);
  }
  c.entry = -1;
  c.nc = 0;
  c.sacc = 0.f;
  c.st = FEMPIC_P_OK;
  c.moved = true;
  c.reflected = false;
}

// Deposit the current piece up to its exit face (or to b) and move on: into
// the neighbour, back from a reflecting wall, or stop (absorbed, capped).
// Returns true when the particle's step is complete.
__device__ __forceinline__ bool cross_advance(const PushArgs& A, CrossState& c, bool fresh) {
  {
    // the current tet's record and the end point's barycentrics in it; a
    // fresh particle also needs its start point's (every busy lane runs this
    // body together, only the start point is particular to fresh lanes)
    const Geo32 G = ld_geo(A.tetrec, c.T);
    FF dd[3];
    float d[3];
    if (fresh) {
      dpos(G, c.a0[0], c.a0[1], c.a0[2], dd, d);
      bary_q(G, d, c.Qa);
    }
    dpos(G, c.b[0], c.b[1], c.b[2], dd, d);
    bary_q(G, d, c.Qb);
  }
  float smin;
  const int kx = exit_face(c.Qa, c.Qb, c.entry, smin);
  long long g[6];
  if (kx < 0) {
    gq(c.Qa, c.Qb, g);
    depositq_atomic(A, c.T, c.s, g);
    return true;
  }
  int32_t Qp[4];
  crossing_q(c.Qa, c.Qb, kx, smin, Qp);
  gq(c.Qa, Qp, g);
  depositq_atomic(A, c.T, c.s, g);
  c.nc++;
  c.sacc = __fmaf_rn(smin, 1.0f - c.sacc, c.sacc);
  if (c.nc > A.max_cross) {
    c.st = FEMPIC_P_CAP;
    c.moved = false;
#pragma unroll
    for (int j = 0; j < 4; j++) c.Qa[j] = Qp[j];   // where the deposited path ends
    return true;
  }
  // neighbour ids from the last 16 B of the tet's record, whose line the
  // walk has just read for the geometry (one round trip less than the
  // separate neighbour table)
  const float4 nbf = __ldg(A.tetrec + 8 * (int64_t)c.T + 7);
  const int4 nbv = make_int4(__float_as_int(nbf.x), __float_as_int(nbf.y), __float_as_int(nbf.z),
                             __float_as_int(nbf.w));
  const int32_t nbt = kx == 0 ? nbv.x : kx == 1 ? nbv.y : kx == 2 ? nbv.z : nbv.w;
  if (nbt >= 0 && !idx_in(nbt, A.nt, A.stats)) {
    c.st = FEMPIC_P_LOST;
    c.moved = false;
#pragma unroll
    for (int j = 0; j < 4; j++) c.Qa[j] = Qp[j];
    return true;
  }
  if (nbt >= 0) {
    // the face map (same record line) says which of this tet's nodes each of
    // the neighbour's nodes is, and which one it enters through
    const float2 fm2 = __ldg(reinterpret_cast<const float2*>(A.tetrec + 8 * (int64_t)c.T + 6) + 1);
    const uint32_t fm = ((kx < 2 ? __float_as_uint(fm2.x) : __float_as_uint(fm2.y)) >> (16 * (kx & 1))) & 0xffffu;
    const int ent = (int)(fm & 3u);
#pragma unroll
    for (int i2 = 0; i2 < 4; i2++) {
      const int j = (int)((fm >> (2 + 2 * i2)) & 3u);
      int32_t val = 0;
#pragma unroll
      for (int jj = 0; jj < 4; jj++)
        if (jj == j) val = Qp[jj];
      c.Qa[i2] = (i2 == ent) ? 0 : val;
    }
    c.T = nbt;
    c.entry = ent;
  } else if (nbt <= -1 && nbt >= -6 && A.wall_mode == FEMPIC_WALL_REFLECT) {
    // materialize the wall point in FP64, mirror the rest of the step
    const double sd = (double)c.sacc;
#pragma unroll
    for (int k = 0; k < 3; k++) c.a0[k] = fma(sd, c.b[k] - c.a0[k], c.a0[k]);
    c.sacc = 0.f;
    const int code = -1 - nbt, ax = code >> 1, side = code & 1;
#pragma unroll
    for (int k = 0; k < 3; k++)
      if (k == ax) {
        const double L = side ? A.hi[k] : A.lo[k];
        c.b[k] = 2.0 * L - c.b[k];
        c.vn[k] = -c.vn[k];
      }
    c.reflected = true;
#pragma unroll
    for (int j = 0; j < 4; j++) c.Qa[j] = Qp[j];
    c.entry = kx;
  } else {
    c.st = FEMPIC_P_ABSORBED;
    c.moved = false;
#pragma unroll
    for (int j = 0; j < 4; j++) c.Qa[j] = Qp[j];   // where the deposited path ends
    return true;
  }
  return false;   // the next call reads the new tet and the end point's barycentrics in it
}

// Final state of a finished walk.
__device__ __forceinline__ void cross_finish(const PushArgs& A, const CrossState& c, unsigned& ncr, unsigned& nfrz) {
  const int64_t p = c.p;
  if (c.moved) {
    if (c.reflected) {   // otherwise b is what the common path already stored
      A.x[p] = c.b[0];
      A.y[p] = c.b[1];
      A.z[p] = c.b[2];
    }
  } else {   // frozen at the last crossing point
    const double sd = (double)c.sacc;
    const double r[3] = {fma(sd, c.b[0] - c.a0[0], c.a0[0]), fma(sd, c.b[1] - c.a0[1], c.a0[1]),
                         fma(sd, c.b[2] - c.a0[2], c.a0[2])};
    A.x[p] = r[0];
    A.y[p] = r[1];
    A.z[p] = r[2];
    // The deposited path ended at the integer crossing point c.Qa, while the
    // particle's charge is assigned from its stored FP64 position; deposit the
    // tiny piece between the two, so that the edge divergence still equals
    // the change of the nodal charge exactly.
    int32_t Qf[4];
    bary_q_at(A.tetrec, c.T, r, Qf);
    long long g[6];
    gq(c.Qa, Qf, g);
    depositq_atomic(A, c.T, c.s, g);
  }
  if (c.reflected) {
    static_cast<float*>(A.vx)[p] = c.vn[0];
    static_cast<float*>(A.vy)[p] = c.vn[1];
    static_cast<float*>(A.vz)[p] = c.vn[2];
  }
  int32_t T = c.T;
  if (c.st != FEMPIC_P_OK) {
    A.status[p] = c.st;
    T = -2 - T;
    nfrz++;
  }
  A.tet[p] = T;
  if (A.ncross) A.ncross[p] += c.nc;
  ncr += (unsigned)c.nc;
}

// Crossing pass of the 24-bit form.  Each warp takes a stream of tile
// regions of the record queue (tile, tile + warps, ...); each loop iteration
// advances every busy lane by one face, and a lane whose particle is done
// takes the stream's next record, so neither a particle that crosses many
// faces (a fast beam particle) nor the end of a tile holds idle lanes.
// Records of one tile come from neighbouring tets, so the warp's tet records
// and deposit slots stay in cache.

__global__ void __launch_bounds__(kThreads) k_cross_q24(PushArgs A, int64_t ntiles) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  unsigned ncr = 0, nfrz = 0;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  int64_t tile = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int32_t cnt = tile < ntiles ? A.xcount[tile] : 0, next = 0;
  bool have = false, fresh = false;
  CrossState c;
  for (;;) {
    unsigned idle = __ballot_sync(full, !have);
    while (idle && tile < ntiles) {   // warp-uniform: assigns records or advances a tile
      const int32_t avail = cnt - next;
      const int32_t want = __popc(idle);
      const int32_t take = avail < want ? avail : want;
      const int r = __popc(idle & lt);
      if (!have && r < take) {
        cross_begin(A, A.xrec[tile * kThreads + next + r], c);
        have = true;
        fresh = true;
      }
      next += take;
      idle = __ballot_sync(full, !have);
      if (next == cnt) {
        tile += warps;
        cnt = tile < ntiles ? A.xcount[tile] : 0;
        next = 0;
      }
    }
    if (!__any_sync(full, have)) break;
    if (have) {
      const bool done = cross_advance(A, c, fresh);
      fresh = false;
      if (done) {
        cross_finish(A, c, ncr, nfrz);
        have = false;
      }
    }
  }
  ncr = __reduce_add_sync(full, ncr);
  nfrz = __reduce_add_sync(full, nfrz);
  if (lane == 0) {
    if (ncr) atomicAdd(A.stats, (unsigned long long)ncr);
    if (nfrz) atomicAdd(A.stats + 1, (unsigned long long)nfrz);
  }
}

// ------------------------------------------- contract-form crossing pass
// The walk of the FP64 oracle (exit face = argmin over the faces with
// lambda_k(b) < 0, entry face excluded, of s_k = lambda_k(a) / (lambda_k(a) -
// lambda_k(b)) clamped at 0, lowest k on ties; crossing barycentrics
// lambda(a) + s (lambda(b) - lambda(a)) with 0 on the exit face; the shared
// nodes' values carried into the neighbour) with every barycentric, every
// exit parameter and every crossing barycentric in double-float, and the
// in-tet pieces deposited in edge form, g_ij = la_i lb_j - la_j lb_i (Sec. II
// eq. g_def), as FP64 atomics of the high parts and FP32 atomics of the low
// parts.  The crossing point itself is FP64 where it is stored (a wall
// reflection, a frozen particle).  GB300 runs FP64 at 1/64 of the FP32 rate,
// so the pass does in FP32 pairs what would otherwise be FP64-pipe bound.
struct CrossStateDF {
  double a0[3], b[3];   // the current straight run goes from a0 to b ...
  DF S;                 // ... and the current piece starts at a0 + S (b - a0)
  FF w[3];              // b - a0 as FP32 pairs (before a reflection: exactly dt v)
  DF la[4];             // barycentrics of the piece start in T
  unsigned flips;       // bit k: velocity component k mirrored an odd number of times
  int32_t T, p;
  int entry, nc, s;
  uint8_t st;
  bool moved, reflected;
};

// lambda(r) in tet T in double-float: d = r - x0 exact in FP64 and split into
// FP32 pairs, lambda_k = (G_k,hi + G_k,lo) . d for k = 1..3 from exact
// products of the high parts, lambda_0 = 1 - lambda_1 - lambda_2 - lambda_3.
__device__ __forceinline__ void lambda_df(const Geo32& G, const float glo[9], const double r[3], DF lam[4],
                                          FF dd[3]) {
  float d32[3];
  dpos(G, r[0], r[1], r[2], dd, d32);
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const float* gh = G.g + 3 * k;
    const float* gl = glo + 3 * k;
    const DF p0 = two_prod(gh[0], dd[0].hi), p1 = two_prod(gh[1], dd[1].hi), p2 = two_prod(gh[2], dd[2].hi);
    const DF s1 = two_sum(p0.h, p1.h);
    const DF s2 = two_sum(s1.h, p2.h);
    float err = __fadd_rn(__fadd_rn(s1.l, s2.l), __fadd_rn(__fadd_rn(p0.l, p1.l), p2.l));
#pragma unroll
    for (int j = 0; j < 3; j++) err = __fmaf_rn(gh[j], dd[j].lo, __fmaf_rn(gl[j], dd[j].hi, err));
    lam[k + 1] = fast_two_sum(s2.h, err);
  }
  lam[0] = df_sub(DF{1.0f, 0.0f}, df_add(df_add(lam[1], lam[2]), lam[3]));
}

__device__ __forceinline__ void ld_glo(const float4* __restrict__ tetdf, int64_t T, float glo[9]) {
  const float4 a = __ldg(tetdf + 4 * T), b = __ldg(tetdf + 4 * T + 1), c = __ldg(tetdf + 4 * T + 2);
  glo[0] = a.x; glo[1] = a.y; glo[2] = a.z; glo[3] = a.w;
  glo[4] = b.x; glo[5] = b.y; glo[6] = b.z; glo[7] = b.w;
  glo[8] = c.x;
}

// Moment-form deposit of the piece of the run a0 -> b between path fractions
// S and S + dS, inside tet T (species s): its displacement dS w and its
// moment about x0, (a0 + S w - x0) x (dS w) = dS ((a0 - x0) x w) (w x w = 0),
// the quantities the common path deposits for a whole segment.  a0 - x0 is
// (b - x0) - w, from the pair the barycentrics of b were formed with.  The
// high FP32 parts go to the FP64 moment slot, the low parts to its FP32
// companion.
__device__ __forceinline__ void deposit_piece_df(const PushArgs& A, int s, int32_t T, const FF w[3],
                                                 const FF db[3], DF dS) {
  if (!A.mom) return;   // deposits off
  DF u[3];
#pragma unroll
  for (int k = 0; k < 3; k++) u[k] = df_sub(DF{db[k].hi, db[k].lo}, DF{w[k].hi, w[k].lo});
  float lo[6];
  double* ms = A.mom + ((int64_t)s * A.nt + T) * 6;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const int i = (k + 1) % 3, j = (k + 2) % 3;   // (u x w)_k = u_i w_j - u_j w_i
    const DF p1 = two_prod(u[i].h, w[j].hi), p2 = two_prod(u[j].h, w[i].hi);
    const DF sd = two_sum(p1.h, -p2.h);
    float e = __fadd_rn(sd.l, __fsub_rn(p1.l, p2.l));
    e = __fmaf_rn(u[i].h, w[j].lo, __fmaf_rn(u[i].l, w[j].hi, e));
    e = __fmaf_rn(-u[j].h, w[i].lo, __fmaf_rn(-u[j].l, w[i].hi, e));
    const DF m = df_mul(dS, fast_two_sum(sd.h, e));
    const DF d = df_mul(dS, DF{w[k].hi, w[k].lo});
    atomicAdd(ms + k, (double)d.h);   // exact widening (the FP64 pipe is idle here)
    atomicAdd(ms + 3 + k, (double)m.h);
    lo[k] = d.l;
    lo[3 + k] = m.l;
  }
  float* ls = A.momlo + ((int64_t)s * A.nt + T) * 8;
  atomicAdd(reinterpret_cast<float4*>(ls), make_float4(lo[0], lo[1], lo[2], lo[3]));
  atomicAdd(reinterpret_cast<float2*>(ls + 4), make_float2(lo[4], lo[5]));
}

__device__ __forceinline__ void cross_begin_df(const PushArgs& A, const CrossRec& r, CrossStateDF& c) {
  c.p = r.p;
  c.T = r.T;
  c.s = species_of(A.sp, r.p);
  const float dt32 = A.dt32;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    c.a0[k] = r.a[k];
    c.w[k] = FF{__fmul_rn(dt32, r.v[k]), 0.f};
    c.b[k] = __dadd_rn(r.a[k], (double)c.w[k].hi);   // advance's value (the widening is exact)
  }
  c.flips = 0u;
  c.S = DF{0.f, 0.f};
  c.entry = -1;
  c.nc = 0;
  c.st = FEMPIC_P_OK;
  c.moved = true;
  c.reflected = false;
}

// The FP64 point a0 + S (b - a0) (a wall point or a frozen particle's stop).
__device__ __forceinline__ void cross_point_df(const CrossStateDF& c, double r[3]) {
  const double sd = df_to_f64(c.S);
#pragma unroll
  for (int k = 0; k < 3; k++) r[k] = fma(sd, c.b[k] - c.a0[k], c.a0[k]);
}

// One piece of the walk: deposit up to the exit face (or to b) and move on.
// Returns true when the particle's step is complete.
__device__ __forceinline__ bool cross_advance_df(const PushArgs& A, CrossStateDF& c, bool fresh) {
  DF lb[4];
  FF db[3];   // b - x0 of this tet
  {
    const Geo32 G = ld_geo(A.tetrec, c.T);
    float glo[9];
    ld_glo(A.tetdf, c.T, glo);
    if (fresh) lambda_df(G, glo, c.a0, c.la, db);
    lambda_df(G, glo, c.b, lb, db);
  }
  int kx = -1;
  DF smin = DF{INFINITY, 0.f};
#pragma unroll
  for (int k = 0; k < 4; k++) {
    if (k == c.entry || !(lb[k].h < 0.f)) continue;
    const DF den = df_sub(c.la[k], lb[k]);
    DF sk = den.h != 0.f ? df_div(c.la[k], den) : DF{0.f, 0.f};
    if (sk.h < 0.f) sk = DF{0.f, 0.f};
    if (df_lt(sk, smin)) {
      smin = sk;
      kx = k;
    }
  }
  const DF rest = df_sub(DF{1.0f, 0.0f}, c.S);   // fraction of the run still ahead
  if (kx < 0) {
    deposit_piece_df(A, c.s, c.T, c.w, db, rest);
    return true;
  }
  DF lp[4];
#pragma unroll
  for (int i = 0; i < 4; i++)
    lp[i] = (i == kx) ? DF{0.f, 0.f} : df_add(c.la[i], df_mul(smin, df_sub(lb[i], c.la[i])));
  const DF dS = df_mul(smin, rest);
  deposit_piece_df(A, c.s, c.T, c.w, db, dS);
  c.nc++;
  c.S = df_add(c.S, dS);
  if (c.nc > A.max_cross) {
    c.st = FEMPIC_P_CAP;
    c.moved = false;
    return true;
  }
  const float4 nbf = __ldg(A.tetrec + 8 * (int64_t)c.T + 7);
  const int4 nbv = make_int4(__float_as_int(nbf.x), __float_as_int(nbf.y), __float_as_int(nbf.z),
                             __float_as_int(nbf.w));
  const int32_t nbt = kx == 0 ? nbv.x : kx == 1 ? nbv.y : kx == 2 ? nbv.z : nbv.w;
  if (nbt >= 0 && !idx_in(nbt, A.nt, A.stats)) {
    c.st = FEMPIC_P_LOST;
    c.moved = false;
    return true;
  }
  if (nbt >= 0) {
    // the face map says which of this tet's nodes each of the neighbour's
    // nodes is, and which one it enters through
    const float2 fm2 = __ldg(reinterpret_cast<const float2*>(A.tetrec + 8 * (int64_t)c.T + 6) + 1);
    const uint32_t fm = ((kx < 2 ? __float_as_uint(fm2.x) : __float_as_uint(fm2.y)) >> (16 * (kx & 1))) & 0xffffu;
    const int ent = (int)(fm & 3u);
#pragma unroll
    for (int i2 = 0; i2 < 4; i2++) {
      const int j = (int)((fm >> (2 + 2 * i2)) & 3u);
      DF val = DF{0.f, 0.f};
#pragma unroll
      for (int jj = 0; jj < 4; jj++)
        if (jj == j) val = lp[jj];
      c.la[i2] = (i2 == ent) ? DF{0.f, 0.f} : val;
    }
    c.T = nbt;
    c.entry = ent;
  } else if (nbt <= -1 && nbt >= -6 && A.wall_mode == FEMPIC_WALL_REFLECT) {
    // the wall point in FP64 starts the mirrored rest of the step
    double wp[3];
    cross_point_df(c, wp);
#pragma unroll
    for (int k = 0; k < 3; k++) c.a0[k] = wp[k];
    c.S = DF{0.f, 0.f};
    const int code = -1 - nbt, ax = code >> 1, side = code & 1;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      if (k == ax) {
        const double L = side ? A.hi[k] : A.lo[k];
        c.b[k] = 2.0 * L - c.b[k];
        c.flips ^= 1u << k;
      }
      c.w[k] = split_f64(__dsub_rn(c.b[k], c.a0[k]));
    }
    c.reflected = true;
#pragma unroll
    for (int j = 0; j < 4; j++) c.la[j] = lp[j];
    c.entry = kx;
  } else {
    c.st = FEMPIC_P_ABSORBED;
    c.moved = false;
    return true;
  }
  return false;
}

__device__ __forceinline__ void cross_finish_df(const PushArgs& A, const CrossStateDF& c, unsigned& ncr,
                                                unsigned& nfrz) {
  const int64_t p = c.p;
  if (!c.moved) {   // frozen at the last crossing point
    double r[3];
    cross_point_df(c, r);
    A.x[p] = r[0];
    A.y[p] = r[1];
    A.z[p] = r[2];
  } else if (c.reflected) {   // otherwise b is what the common path already stored
    A.x[p] = c.b[0];
    A.y[p] = c.b[1];
    A.z[p] = c.b[2];
  }
  // the common path stored the new velocity; mirror the reflected components
  float* vv[3] = {static_cast<float*>(A.vx), static_cast<float*>(A.vy), static_cast<float*>(A.vz)};
#pragma unroll
  for (int k = 0; k < 3; k++)
    if (c.flips & (1u << k)) vv[k][p] = -vv[k][p];
  int32_t T = c.T;
  if (c.st != FEMPIC_P_OK) {
    A.status[p] = c.st;
    T = -2 - T;
    nfrz++;
  }
  A.tet[p] = T;
  if (A.ncross) A.ncross[p] += c.nc;
  ncr += (unsigned)c.nc;
}

// Each loop iteration advances every busy lane by one piece; idle lanes take
// the next records of the warp's record stream, which runs on across its
// tiles (tile, tile + warps, ...): a tile holds about 36 leaving particles
// on the cavity, so a per-tile loop would leave most lanes idle at the end of
// every tile (the stream measured 9 % faster).
#ifndef FEMPIC_CROSS_MIN_BLOCKS
#define FEMPIC_CROSS_MIN_BLOCKS 3
#endif
__global__ void __launch_bounds__(kThreads, FEMPIC_CROSS_MIN_BLOCKS) k_cross_df(PushArgs A, int64_t ntiles) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  unsigned ncr = 0, nfrz = 0;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  int64_t tile = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int32_t cnt = tile < ntiles ? A.xcount[tile] : 0, next = 0;
  bool have = false, fresh = false;
  CrossStateDF c;
  for (;;) {
    unsigned idle = __ballot_sync(full, !have);
    while (idle && tile < ntiles) {   // warp-uniform: assigns records or advances a tile
      const int32_t avail = cnt - next;
      const int32_t want = __popc(idle);
      const int32_t take = avail < want ? avail : want;
      const int r = __popc(idle & lt);
      if (!have && r < take) {
        cross_begin_df(A, A.xrec[tile * kThreads + next + r], c);
        have = true;
        fresh = true;
      }
      next += take;
      idle = __ballot_sync(full, !have);
      if (next == cnt) {
        tile += warps;
        cnt = tile < ntiles ? A.xcount[tile] : 0;
        next = 0;
      }
    }
    if (!__any_sync(full, have)) break;
    if (have) {
      const bool done = cross_advance_df(A, c, fresh);
      fresh = false;
      if (done) {
        cross_finish_df(A, c, ncr, nfrz);
        have = false;
      }
    }
  }
  ncr = __reduce_add_sync(full, ncr);
  nfrz = __reduce_add_sync(full, nfrz);
  if (lane == 0) {
    if (ncr) atomicAdd(A.stats, (unsigned long long)ncr);
    if (nfrz) atomicAdd(A.stats + 1, (unsigned long long)nfrz);
  }
}

// ------------------------------------------------------- deposit finalize
// Contract form, per tet: the moment slots (sum of D, sum of u x D, FP64)
// become the 6 local-edge values through the tet's gradients,
//   g_0j = G_j . sum D + (G_0 x G_j) . sum(u x D),  g_ij = (G_i x G_j) . sum(u x D),
// in double-float from the FP64 gradients' FP32 pairs; the crossing pass's
// edge-form deposits are added, each species scaled by its q w, and the sum
// is written as FP32 pairs for the per-edge pull.  The slots are cleared.
struct TetFinalizeArgs {
  int64_t nt;
  int32_t ns;
  const float4* tetrec;
  const float4* tetdf;
  double* mom;
  float* momlo;
  float qwh[kMaxSpecies], qwl[kMaxSpecies];   // q w per species as FP32 pairs
  float4* out;                                // [nt][3]: (h, l) of local edges 0..5
};

__device__ __forceinline__ void df_cross(const DF a[3], const DF b[3], DF c[3]) {
  c[0] = df_sub(df_mul(a[1], b[2]), df_mul(a[2], b[1]));
  c[1] = df_sub(df_mul(a[2], b[0]), df_mul(a[0], b[2]));
  c[2] = df_sub(df_mul(a[0], b[1]), df_mul(a[1], b[0]));
}

__global__ void __launch_bounds__(kThreads) k_tet_finalize(TetFinalizeArgs A) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= A.nt) return;
  // the slots' sums, as FP32 pairs, scaled by q w and summed over species
  // (the conversion below is linear in them)
  DF S[3] = {DF{0.f, 0.f}, DF{0.f, 0.f}, DF{0.f, 0.f}}, M[3] = {DF{0.f, 0.f}, DF{0.f, 0.f}, DF{0.f, 0.f}};
  bool any = false;
  for (int s = 0; s < A.ns; s++) {
    double2* m2 = reinterpret_cast<double2*>(A.mom + ((int64_t)s * A.nt + t) * 6);
    float4* l4 = reinterpret_cast<float4*>(A.momlo + ((int64_t)s * A.nt + t) * 8);
    const double2 a = m2[0], b = m2[1], c = m2[2];
    const float4 la = l4[0], lb = l4[1];
    const double mv[6] = {a.x, a.y, b.x, b.y, c.x, c.y};
    const float lv[6] = {la.x, la.y, la.z, la.w, lb.x, lb.y};
    bool here = false;
#pragma unroll
    for (int e = 0; e < 6; e++) here = here || mv[e] != 0.0 || lv[e] != 0.f;
    if (!here) continue;
    any = true;
    const double2 z2 = make_double2(0.0, 0.0);
    m2[0] = m2[1] = m2[2] = z2;
    l4[0] = l4[1] = make_float4(0.f, 0.f, 0.f, 0.f);
    const DF qw = DF{A.qwh[s], A.qwl[s]};
#pragma unroll
    for (int k = 0; k < 3; k++) {
      S[k] = df_add(S[k], df_mul(qw, df_add(f64_to_df(mv[k]), DF{lv[k], 0.f})));
      M[k] = df_add(M[k], df_mul(qw, df_add(f64_to_df(mv[3 + k]), DF{lv[3 + k], 0.f})));
    }
  }
  float4* o = A.out + 3 * t;
  if (!any) {
    o[0] = o[1] = o[2] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  // gradients G_1..3 as FP32 pairs, G_0 = -(G_1 + G_2 + G_3)
  const float4 a = __ldg(A.tetrec + 8 * t + 1), b = __ldg(A.tetrec + 8 * t + 2), c = __ldg(A.tetrec + 8 * t + 3);
  const float4 p = __ldg(A.tetdf + 4 * t), q = __ldg(A.tetdf + 4 * t + 1), r = __ldg(A.tetdf + 4 * t + 2);
  const float gh[9] = {a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z};
  const float gl[9] = {p.x, p.y, p.z, p.w, q.x, q.y, q.z, q.w, r.x};
  DF G[4][3];
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int j = 0; j < 3; j++) G[k + 1][j] = fast_two_sum(gh[3 * k + j], gl[3 * k + j]);
#pragma unroll
  for (int j = 0; j < 3; j++) G[0][j] = df_neg(df_add(df_add(G[1][j], G[2][j]), G[3][j]));
  DF g[6];
#pragma unroll
  for (int e = 0; e < 6; e++) {
    const int i = le0(e), j = le1(e);
    DF C[3];
    df_cross(G[i], G[j], C);
    g[e] = df_dot3(C, M);
    if (i == 0) g[e] = df_add(g[e], df_dot3(G[j], S));
  }
  o[0] = make_float4(g[0].h, g[0].l, g[1].h, g[1].l);
  o[1] = make_float4(g[2].h, g[2].l, g[3].h, g[3].l);
  o[2] = make_float4(g[4].h, g[4].l, g[5].h, g[5].l);
}

struct FinalizeArgs {
  int64_t ne;
  int64_t nt;
  const int32_t* estart;         // mixed forms: edge -> (tet, local edge) slots
  const int32_t* eslot;
  int32_t mode;                  // 0 FP64 accumulator, 1 contract form (per-tet pairs), 2 24-bit form
  int32_t ns;
  double qwscale[kMaxSpecies];   // q w 2^-48 per species (24-bit form)
  double* dG;
  const unsigned long long* dGq;  // 24-bit form: deposit slots [ns][nt][8]
  const float* tetout;           // contract form: [nt][12] (h, l) pairs of the 6 local edges
  double* Gcum;
  double* dG_out;
  double* Gcum_out;
  double2* Genv_out;
  double c, s;                   // cos, sin of omega0 t_next
  int32_t local;                 // 1: write dG_out only, leave G_cum (fempic_deposit_local)
  unsigned long long* stats;     // bounds checks of the debug build
};

// Deposit finalize, one thread per edge.  The mixed forms pull the edge's
// values from its tets (adjacency built once on the host, a fixed order):
// the 24-bit form its exact int64 sums from the integer slots, scaled by
// q w 2^-48 (the slots are cleared afterwards by one coalesced memset); the
// contract form its tets' double-float values from k_tet_finalize.  FP64
// form: the edge's FP64 accumulator.  Then G_cum += dG and the requested
// outputs (dG, G_cum, the envelope-frame G~).
__global__ void __launch_bounds__(kThreads) k_deposit_finalize(FinalizeArgs A) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= A.ne) return;
  double d;
  if (A.mode == 2) {
    d = 0.0;
    const int32_t j0 = A.estart[e], j1 = A.estart[e + 1];
    for (int s = 0; s < A.ns; s++) {
      long long q = 0;
      const unsigned long long* sl = A.dGq + (int64_t)s * A.nt * 8;
      for (int32_t j = j0; j < j1; j++) {
        const int32_t k = A.eslot[j];
        if (idx_in(k, 6 * A.nt, A.stats)) q += (long long)sl[(int64_t)(k / 6) * 8 + k % 6];
      }
      d += A.qwscale[s] * (double)q;
    }
  } else if (A.mode == 1) {
    DF acc = DF{0.f, 0.f};
    const int32_t j0 = A.estart[e], j1 = A.estart[e + 1];
    for (int32_t j = j0; j < j1; j++) {
      const int32_t k = A.eslot[j];
      if (!idx_in(k, 6 * A.nt, A.stats)) continue;
      const float2 v = reinterpret_cast<const float2*>(A.tetout)[(int64_t)(k / 6) * 6 + k % 6];
      acc = df_add(acc, DF{v.x, v.y});
    }
    d = df_to_f64(acc);
  } else {
    d = A.dG[e];
    A.dG[e] = 0.0;
  }
  if (A.local) {
    A.dG_out[e] = d;
    return;
  }
  const double g = A.Gcum[e] + d;
  A.Gcum[e] = g;
  if (A.dG_out) A.dG_out[e] = d;
  if (A.Gcum_out) A.Gcum_out[e] = g;
  if (A.Genv_out) A.Genv_out[e] = make_double2(A.c * g, -(A.s * g));
}

// G_cum += dG for a step deposit reduced outside the library (a sharded run
// all-reduces each rank's dG), then the requested outputs.
__global__ void __launch_bounds__(kThreads) k_accumulate(int64_t ne, const double* __restrict__ dG,
                                                         double* __restrict__ Gcum, double* Gcum_out,
                                                         double2* Genv_out, double c, double s) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const double g = Gcum[e] + dG[e];
  Gcum[e] = g;
  if (Gcum_out) Gcum_out[e] = g;
  if (Genv_out) Genv_out[e] = make_double2(c * g, -(s * g));
}

// ------------------------------------------------------------ nodal charge
struct ChargeArgs {
  int64_t n;
  const double* x;
  const double* y;
  const double* z;
  const int32_t* tet;
  Species sp;
  int64_t nt;
  int32_t q24;                // 24-bit form: the integer barycentrics its deposit uses
  const double* geom64;
  const float4* tetrec;
  const int4* tn;
  double* rho;
  int64_t nn;                 // node count and stats: bounds checks of the debug build
  unsigned long long* stats;
};

__global__ void __launch_bounds__(kThreads) k_nodal_charge(ChargeArgs A) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= A.n) return;
  int32_t T = A.tet[p];
  if (T == -1) return;
  if (T < 0) T = -2 - T;
  if (T >= A.nt) return;
  const int s = species_of(A.sp, p);
  const double qw = A.sp.qw[s];
  const double r[3] = {A.x[p], A.y[p], A.z[p]};
  double lam[4];
  if (A.q24) {
    int32_t Q[4];
    bary_q_at(A.tetrec, T, r, Q);
    for (int i = 0; i < 4; i++) lam[i] = (double)Q[i] * (1.0 / (double)kQOne);
  } else {
    bary64(A.geom64 + 12 * (int64_t)T, r, lam);
  }
  const int4 n4 = A.tn[T];
  const int32_t nid[4] = {n4.x, n4.y, n4.z, n4.w};
#pragma unroll
  for (int i = 0; i < 4; i++)
    if (idx_in(nid[i], A.nn, A.stats)) atomicAdd(A.rho + nid[i], qw * lam[i]);
}


// ------------------------------------------------------------ particle sort
// Counting sort by key = species * (nt + 1) + (0 <= tet < nt ? tet : nt).
__device__ __forceinline__ int32_t sort_key(const Species& sp, int64_t p, int32_t T, int64_t nt) {
  const int s = species_of(sp, p);
  return (int32_t)(s * (nt + 1) + ((T >= 0 && T < nt) ? (int64_t)T : nt));
}

__global__ void __launch_bounds__(kThreads) k_sort_hist(int64_t n, const int32_t* __restrict__ tet, Species sp,
                                                         int64_t nt, int32_t* __restrict__ counts) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool act = p < n;
  const int32_t key = act ? sort_key(sp, p, tet[p], nt) : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int lane = threadIdx.x & 31;
  if (act && lane == __ffs(peers) - 1) atomicAdd(counts + key, __popc(peers));
}

// Exclusive scan over `k` int32 counts in tiles of 2 * kScan; tile totals go
// to `sums`, scanned by one block, then added back.
constexpr int kScan = 1024;

__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t* sh, int32_t* total) {
  // Hillis-Steele inclusive scan in shared memory over blockDim.x entries
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int off = 1; off < blockDim.x; off <<= 1) {
    const int32_t o = t >= off ? sh[t - off] : 0;
    __syncthreads();
    sh[t] += o;
    __syncthreads();
  }
  const int32_t incl = sh[t];
  *total = sh[blockDim.x - 1];
  __syncthreads();
  return incl - v;
}

__global__ void __launch_bounds__(kScan) k_scan_tiles(int64_t k, const int32_t* __restrict__ in,
                                                      int32_t* __restrict__ out, int32_t* __restrict__ sums) {
  __shared__ int32_t sh[kScan];
  const int64_t base = blockIdx.x * (int64_t)(2 * kScan);
  const int64_t i0 = base + 2 * threadIdx.x;
  const int32_t a = i0 < k ? in[i0] : 0, b = i0 + 1 < k ? in[i0 + 1] : 0;
  int32_t total;
  const int32_t ex = block_excl_scan(a + b, sh, &total);
  if (i0 < k) out[i0] = ex;
  if (i0 + 1 < k) out[i0 + 1] = ex + a;
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScan) k_scan_sums(int64_t m, int32_t* __restrict__ sums) {
  __shared__ int32_t sh[kScan];
  int32_t carry = 0;
  for (int64_t c = 0; c < m; c += kScan) {
    const int64_t i = c + threadIdx.x;
    const int32_t v = i < m ? sums[i] : 0;
    int32_t total;
    const int32_t ex = block_excl_scan(v, sh, &total);
    if (i < m) sums[i] = carry + ex;
    carry += total;
  }
}

__global__ void __launch_bounds__(kThreads) k_scan_add(int64_t k, int32_t* __restrict__ out,
                                                        const int32_t* __restrict__ sums) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < k) out[i] += sums[i / (2 * kScan)];
}

struct SortArgs {
  int64_t n;
  Species sp;
  int64_t nt;
  int32_t vbytes;               // 8 (FP64 form) or 4 (mixed)
  const double *x, *y, *z;
  const void *vx, *vy, *vz;
  const int32_t* tet;
  const uint8_t* status;
  const int32_t* ncross;
  double *ox, *oy, *oz;
  void *ovx, *ovy, *ovz;
  int32_t* otet;
  uint8_t* ostatus;
  int32_t* oncross;
  const int32_t* offsets;
  int32_t* cursor;
  int32_t* operm;               // optional: source index of each output position
};

__global__ void __launch_bounds__(kThreads) k_sort_scatter(SortArgs A) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool act = p < A.n;
  const int32_t T = act ? A.tet[p] : 0;
  const int32_t key = act ? sort_key(A.sp, p, T, A.nt) : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  int32_t base = 0;
  if (act && lane == leader) base = atomicAdd(A.cursor + key, __popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (!act) return;
  const int64_t q = (int64_t)A.offsets[key] + base + __popc(peers & ((1u << lane) - 1u));
  A.ox[q] = A.x[p];
  A.oy[q] = A.y[p];
  A.oz[q] = A.z[p];
  if (A.vbytes == 8) {
    static_cast<double*>(A.ovx)[q] = static_cast<const double*>(A.vx)[p];
    static_cast<double*>(A.ovy)[q] = static_cast<const double*>(A.vy)[p];
    static_cast<double*>(A.ovz)[q] = static_cast<const double*>(A.vz)[p];
  } else {
    static_cast<float*>(A.ovx)[q] = static_cast<const float*>(A.vx)[p];
    static_cast<float*>(A.ovy)[q] = static_cast<const float*>(A.vy)[p];
    static_cast<float*>(A.ovz)[q] = static_cast<const float*>(A.vz)[p];
  }
  A.otet[q] = T;
  A.ostatus[q] = A.status[p];
  if (A.oncross) A.oncross[q] = A.ncross[p];
  if (A.operm) A.operm[q] = (int32_t)p;
}

// Adjoint state carried back across a sort: out[perm[q]] = in[q].
struct AdjPermArgs {
  int64_t n;
  int32_t vbytes;
  const int32_t* perm;
  const double *rx, *ry, *rz;
  const void *vx, *vy, *vz;
  double *ox, *oy, *oz;
  void *ovx, *ovy, *ovz;
};

__global__ void __launch_bounds__(kThreads) k_adjoint_unpermute(AdjPermArgs A) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= A.n) return;
  const int64_t p = A.perm[q];
  if (p < 0 || p >= A.n) return;   // not a permutation of 0..n-1: leave the slot (checked on the host side too)
  A.ox[p] = A.rx[q];
  A.oy[p] = A.ry[q];
  A.oz[p] = A.rz[q];
  if (A.vbytes == 8) {
    static_cast<double*>(A.ovx)[p] = static_cast<const double*>(A.vx)[q];
    static_cast<double*>(A.ovy)[p] = static_cast<const double*>(A.vy)[q];
    static_cast<double*>(A.ovz)[p] = static_cast<const double*>(A.vz)[q];
  } else {
    static_cast<float*>(A.ovx)[p] = static_cast<const float*>(A.vx)[q];
    static_cast<float*>(A.ovy)[p] = static_cast<const float*>(A.vy)[q];
    static_cast<float*>(A.ovz)[p] = static_cast<const float*>(A.vz)[q];
  }
}

// ----------------------------------------------------------------- adjoint
// Reverse mode of one particle step for the fixed tet sequence of the forward
// step.  Per particle it recomputes the gather and the Boris rotation from
// the state before the step, reads which walls mirrored the particle from
// the sign of each velocity component after the step, and propagates the
// adjoint (rbar, vbar) of the state after the step back to the state before
// it.  The adjoint of the per-tet affine field (E0, W, B0, beta) is reduced
// over runs of equal tets in each warp and added per tet: in FP64 (FP64
// form) or into an FP32 row with vector atomics (mixed form, no FP64-pipe
// work); in the mixed form a warp whose particles fall into more than 4 runs
// (the order has drifted since the last sort) skips the reduction and adds
// each lane's 10 values straight into the row.  The transposed pre-pass k_field_adjoint maps both
// to the complex DoFs.  A
// particle frozen during the step gets a zero adjoint (its later state no
// longer depends on its earlier one through the step map).
struct AdjArgs {
  int64_t n;
  const double* x;
  const double* y;
  const double* z;
  const void* vx;
  const void* vy;
  const void* vz;
  const int32_t* tet;
  const void* vx1;           // velocities after the step
  const void* vy1;
  const void* vz1;
  const uint8_t* status1;    // statuses after the step
  Species sp;
  double dt;
  int64_t nt;
  const double* geom64;
  const double* field64;
  const float4* tetrec;
  double* rbx;
  double* rby;
  double* rbz;
  void* vbx;
  void* vby;
  void* vbz;
  double* tetgrad;           // [nt][10]
  float* tetgrad32;          // mixed form: [nt][12] (10 used), per-lane vector atomics
  // deposited-current loss (fempic_adjoint_current_weights): per-tet alpha, beta [nt][6], or NULL
  const double* curw;
  const int4* nb;
  const int4* tn;
  unsigned long long* stats;   // bounds checks of the debug build
  int32_t max_cross;
  int32_t wall_mode;
  double lo[3], hi[3];
};

// ------------------------------------------------ adjoint of the deposit
// Loss L = sum_e u_e dG_e over the step's deposit.  Inside a tet the
// deposit of a straight piece p -> q is linear in (q - p) and in the moment
// (p - x0) x (q - p) (g_0j = G_j . D + (G_0 x G_j) . M, g_ij = (G_i x G_j) .
// M), so its share of L is alpha . (q - p) + beta . ((p - x0) x (q - p))
// with the per-tet vectors alpha = sum_j u_0j G_j and beta = sum_e u_e
// (G_i x G_j) (k_current_weights).  The gradient of one particle's share
// with respect to its start a and displacement w (the straight run a -> a +
// w) follows the FP64 walk again: a crossing point q = a0 + S w on face f
// moves in the face plane, dq = P (da0 + S dw) with P = I - w G_f^T / (G_f .
// w); a wall reflection starts a new run a0' = q, w' = M (1 - S) w (M the
// mirror), whose Jacobian is folded into the running 6 x 6 one.
__device__ __forceinline__ void cross3d(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ double dot3d(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Gradient rows of tet T (FP64): G[k] = grad lambda_k, G_0 = -(G_1 + G_2 + G_3).
__device__ __forceinline__ void grads64(const double* geom64, int32_t T, double G[4][3]) {
  const double* g = geom64 + 12 * (int64_t)T;
#pragma unroll
  for (int k = 1; k < 4; k++)
#pragma unroll
    for (int c = 0; c < 3; c++) G[k][c] = g[3 * k + c];
#pragma unroll
  for (int c = 0; c < 3; c++) G[0][c] = -((G[1][c] + G[2][c]) + G[3][c]);
}

// d(loss)/d(a), d(loss)/d(w) of one particle-step whose run starts at a with
// end b (= a + w as the forward step formed it), tet T0 at the start.
// The 6 x 6 Jacobian lives in local memory (loops not unrolled): only
// particles that reflected in this step touch it.
__device__ __noinline__ void dep_loss_grad(const AdjArgs& A, int32_t T0, const double a[3], const double b_in[3],
                                           double ga[3], double gw[3]) {
  double a0[3], b[3], w[3], pnt[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    a0[c] = a[c];
    b[c] = b_in[c];
    w[c] = b[c] - a[c];
    pnt[c] = a[c];
    ga[c] = gw[c] = 0.0;
  }
  double J[6][6];          // d(a0, w of the current run) / d(a, w of the step), once a wall reflected it
  bool refl = false;
  double gprev[3] = {0.0, 0.0, 0.0}, Sprev = 0.0;
  bool on_face = false;    // the piece start is a crossing point of this run (face gradient gprev)
  double S = 0.0;
  int32_t T = T0;
  int entry = -1, nc = 0;
  double la[4], lb[4];
  bary64(A.geom64 + 12 * (int64_t)T, pnt, la);
  for (;;) {
    bary64(A.geom64 + 12 * (int64_t)T, b, lb);
    int kx = -1;
    double smin = INFINITY;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      if (k == entry || !negative_bits(lb[k])) continue;
      double sk = la[k] / (la[k] - lb[k]);
      if (sk < 0.0) sk = 0.0;
      if (sk < smin) {
        smin = sk;
        kx = k;
      }
    }
    double G[4][3];
    grads64(A.geom64, T, G);
    const double* cw = A.curw + 6 * (int64_t)T;
    const double al[3] = {cw[0], cw[1], cw[2]}, be[3] = {cw[3], cw[4], cw[5]};
    const double* x0 = A.geom64 + 12 * (int64_t)T;
    double q[3], Sq = 1.0;
    if (kx < 0) {
#pragma unroll
      for (int c = 0; c < 3; c++) q[c] = b[c];
    } else {
#pragma unroll
      for (int c = 0; c < 3; c++) q[c] = fma(smin, b[c] - pnt[c], pnt[c]);
      Sq = S + smin * (1.0 - S);
    }
    // this piece's gradients at its ends
    double u[3], d[3], bu[3], db_[3], gp[3], gq[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      u[c] = pnt[c] - x0[c];
      d[c] = q[c] - pnt[c];
    }
    cross3d(be, u, bu);
    cross3d(d, be, db_);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      gp[c] = -al[c] - bu[c] + db_[c];
      gq[c] = al[c] + bu[c];
    }
    // ... through the ends' dependence on (a0, w) of this run
    double ca[3], cwv[3];
    {
      double tp[3];
      if (on_face) {
        const double f = dot3d(w, gp) / dot3d(gprev, w);
#pragma unroll
        for (int c = 0; c < 3; c++) tp[c] = gp[c] - gprev[c] * f;
      } else {
#pragma unroll
        for (int c = 0; c < 3; c++) tp[c] = gp[c];
      }
#pragma unroll
      for (int c = 0; c < 3; c++) {
        ca[c] = tp[c];
        cwv[c] = on_face ? Sprev * tp[c] : 0.0;
      }
      if (kx < 0) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
          ca[c] += gq[c];
          cwv[c] += gq[c];
        }
      } else {
        const double f = dot3d(w, gq) / dot3d(G[kx], w);
#pragma unroll
        for (int c = 0; c < 3; c++) {
          const double t = gq[c] - G[kx][c] * f;
          ca[c] += t;
          cwv[c] += Sq * t;
        }
      }
    }
    // ... and through the run's dependence on the step's (a, w)
    if (refl) {
#pragma unroll 1
      for (int i = 0; i < 3; i++) {
        double sa = 0.0, sw = 0.0;
#pragma unroll
        for (int r = 0; r < 3; r++) {
          sa += J[r][i] * ca[r] + J[3 + r][i] * cwv[r];
          sw += J[r][3 + i] * ca[r] + J[3 + r][3 + i] * cwv[r];
        }
        ga[i] += sa;
        gw[i] += sw;
      }
    } else {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        ga[c] += ca[c];
        gw[c] += cwv[c];
      }
    }
    if (kx < 0) break;
    double lp[4];
#pragma unroll
    for (int i = 0; i < 4; i++) lp[i] = (i == kx) ? 0.0 : fma(smin, lb[i] - la[i], la[i]);
    nc++;
    if (nc > A.max_cross) break;   // frozen at q: the deposit ended there
    const int4 nbv = ldg_int4(&A.nb[T]);
    const int32_t nbt = kx == 0 ? nbv.x : kx == 1 ? nbv.y : kx == 2 ? nbv.z : nbv.w;
    if (nbt >= 0 && !idx_in(nbt, A.nt, A.stats)) break;
    if (nbt >= 0) {
      const int4 o4 = ldg_int4(&A.tn[T]), n4 = ldg_int4(&A.tn[nbt]);
      const int32_t on[4] = {o4.x, o4.y, o4.z, o4.w}, nn[4] = {n4.x, n4.y, n4.z, n4.w};
      int ent = 0;
#pragma unroll
      for (int i2 = 0; i2 < 4; i2++) {
        int hit = -1;
#pragma unroll
        for (int i = 0; i < 4; i++)
          if (on[i] == nn[i2]) hit = i;
        double val = 0.0;
#pragma unroll
        for (int i = 0; i < 4; i++)
          if (i == hit) val = lp[i];
        la[i2] = val;
        if (hit < 0) ent = i2;
      }
#pragma unroll
      for (int c = 0; c < 3; c++) {
        gprev[c] = G[kx][c];
        pnt[c] = q[c];
      }
      Sprev = Sq;
      S = Sq;
      on_face = true;
      T = nbt;
      entry = ent;
    } else if (nbt <= -1 && nbt >= -6 && A.wall_mode == FEMPIC_WALL_REFLECT) {
      // new run a0' = q, w' = M (1 - Sq) w: its Jacobian with respect to this run
      const int code = -1 - nbt, ax = code >> 1, side = code & 1;
      const double gfw = dot3d(G[kx], w);
      double Jr[6][6];
#pragma unroll 1
      for (int i = 0; i < 3; i++)
#pragma unroll 1
        for (int j = 0; j < 3; j++) {
          const double pij = (i == j ? 1.0 : 0.0) - w[i] * G[kx][j] / gfw;   // P = I - w G_f^T / (G_f . w)
          const double mi = (i == ax) ? -1.0 : 1.0;
          Jr[i][j] = pij;
          Jr[i][3 + j] = Sq * pij;
          Jr[3 + i][j] = mi * w[i] * G[kx][j] / gfw;
          Jr[3 + i][3 + j] = mi * ((i == j ? 1.0 - Sq : 0.0) + Sq * w[i] * G[kx][j] / gfw);
        }
      if (refl) {
        double Jn[6][6];
#pragma unroll 1
        for (int i = 0; i < 6; i++)
#pragma unroll 1
          for (int j = 0; j < 6; j++) {
            double acc = 0.0;
#pragma unroll 1
            for (int k = 0; k < 6; k++) acc += Jr[i][k] * J[k][j];
            Jn[i][j] = acc;
          }
#pragma unroll 1
        for (int i = 0; i < 36; i++) J[i / 6][i % 6] = Jn[i / 6][i % 6];
      } else {
#pragma unroll 1
        for (int i = 0; i < 36; i++) J[i / 6][i % 6] = Jr[i / 6][i % 6];
        refl = true;
      }
      const double L = side ? A.hi[ax] : A.lo[ax];
      b[ax] = 2.0 * L - b[ax];
#pragma unroll
      for (int c = 0; c < 3; c++) {
        a0[c] = q[c];
        pnt[c] = q[c];
        w[c] = b[c] - a0[c];
      }
#pragma unroll
      for (int i = 0; i < 4; i++) la[i] = lp[i];
      entry = kx;
      S = 0.0;
      on_face = false;
    } else {
      break;   // absorbed at q
    }
  }
}

template <typename R>
struct Vec {
  R x, y, z;
};
template <typename R>
__device__ __forceinline__ Vec<R> vx3(Vec<R> a, Vec<R> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename R>
__device__ __forceinline__ R vd3(Vec<R> a, Vec<R> b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}

__device__ __forceinline__ double flip_sign(double x, bool neg) {
  return __hiloint2double(__double2hiint(x) ^ (neg ? (int)0x80000000 : 0), __double2loint(x));
}
__device__ __forceinline__ double widen(float x) { return f32_to_f64(x); }
__device__ __forceinline__ double widen(double x) { return x; }

template <typename R, bool DEP>
__device__ __forceinline__ void adjoint_particle(const AdjArgs& A, int64_t p, int32_t T, R out[10]) {
  const int s = species_of(A.sp, p);
  const R kq = (R)A.sp.kq[s];
  const R* vx = static_cast<const R*>(A.vx);
  const R* vy = static_cast<const R*>(A.vy);
  const R* vz = static_cast<const R*>(A.vz);
  const Vec<R> v = {vx[p], vy[p], vz[p]};
  Vec<R> d, E0, W, B0;
  R beta;
  if (sizeof(R) == 8) {
    const double* G = A.geom64 + 12 * (int64_t)T;
    const double* F = A.field64 + 10 * (int64_t)T;
    d = {(R)(A.x[p] - G[0]), (R)(A.y[p] - G[1]), (R)(A.z[p] - G[2])};
    E0 = {(R)F[0], (R)F[1], (R)F[2]};
    W = {(R)F[3], (R)F[4], (R)F[5]};
    B0 = {(R)F[6], (R)F[7], (R)F[8]};
    beta = (R)F[9];
  } else {
    const float4* Rr = A.tetrec + 8 * (int64_t)T;
    const Geo32 G = ld_geo(A.tetrec, T);
    const float4 f0 = __ldg(Rr + 4), f1 = __ldg(Rr + 5), f2 = __ldg(Rr + 6);
    FF dd[3];
    float d32[3];
    dpos(G, A.x[p], A.y[p], A.z[p], dd, d32);   // the forward step's sequence
    d = {(R)d32[0], (R)d32[1], (R)d32[2]};
    E0 = {(R)f0.x, (R)f0.y, (R)f0.z};
    W = {(R)f0.w, (R)f1.x, (R)f1.y};
    B0 = {(R)f1.z, (R)f1.w, (R)f2.x};
    beta = (R)f2.y;
  }
  // forward recompute
  const Vec<R> dW = vx3(d, W);
  const Vec<R> E = {E0.x + dW.x, E0.y + dW.y, E0.z + dW.z};
  const Vec<R> B = {B0.x + beta * d.x, B0.y + beta * d.y, B0.z + beta * d.z};
  const Vec<R> vm = {v.x + kq * E.x, v.y + kq * E.y, v.z + kq * E.z};
  const Vec<R> tau = {kq * B.x, kq * B.y, kq * B.z};
  const R t2 = vd3(tau, tau);
  const R f = R(2) / (R(1) + t2);
  const Vec<R> sv = {f * tau.x, f * tau.y, f * tau.z};
  const Vec<R> c1 = vx3(vm, tau);
  const Vec<R> vp = {vm.x + c1.x, vm.y + c1.y, vm.z + c1.z};
  const Vec<R> c2 = vx3(vp, sv);
  const Vec<R> vn = {vm.x + c2.x + kq * E.x, vm.y + c2.y + kq * E.y, vm.z + c2.z + kq * E.z};
  // wall mirrors: a reflected component comes out with the opposite sign
  const R* vx1 = static_cast<const R*>(A.vx1);
  const R* vy1 = static_cast<const R*>(A.vy1);
  const R* vz1 = static_cast<const R*>(A.vz1);
  const R mx = vn.x * vx1[p] < R(0) ? R(-1) : R(1);
  const R my = vn.y * vy1[p] < R(0) ? R(-1) : R(1);
  const R mz = vn.z * vz1[p] < R(0) ? R(-1) : R(1);
  R* vbx = static_cast<R*>(A.vbx);
  R* vby = static_cast<R*>(A.vby);
  R* vbz = static_cast<R*>(A.vbz);
  // adjoint of the output state, mirrored back (sign flips on the bit pattern)
  const double rbx = flip_sign(A.rbx[p], mx < R(0)), rby = flip_sign(A.rby[p], my < R(0)),
               rbz = flip_sign(A.rbz[p], mz < R(0));
  const R dt = (R)A.dt;
  // b = r + dt vn
  Vec<R> vnb = {mx * vbx[p] + dt * (R)rbx, my * vby[p] + dt * (R)rby, mz * vbz[p] + dt * (R)rbz};
  double dga[3] = {0.0, 0.0, 0.0};
  if (DEP) {   // this step's share of the deposited-current loss, through a and w = dt vn
    const double a[3] = {A.x[p], A.y[p], A.z[p]};
    const R vf[3] = {mx * vx1[p], my * vy1[p], mz * vz1[p]};   // the forward's vn, exactly
    double b[3], gw[3];
#pragma unroll
    for (int c = 0; c < 3; c++)
      b[c] = sizeof(R) == 8 ? fma(A.dt, (double)vf[c], a[c]) : advance(a[c], (float)A.dt, (float)vf[c]);
    dep_loss_grad(A, T, a, b, dga, gw);
    const double qw = A.sp.qw[s];
    vnb.x += (R)(A.dt * qw * gw[0]);
    vnb.y += (R)(A.dt * qw * gw[1]);
    vnb.z += (R)(A.dt * qw * gw[2]);
#pragma unroll
    for (int c = 0; c < 3; c++) dga[c] *= qw;
  }
  // vn = vpl + kq E ;  vpl = vm + vp x s
  Vec<R> Eb = {kq * vnb.x, kq * vnb.y, kq * vnb.z};
  Vec<R> vmb = vnb;
  const Vec<R> vpb = vx3(sv, vnb);
  const Vec<R> sb = vx3(vnb, vp);
  // s = f tau
  Vec<R> taub = {f * sb.x, f * sb.y, f * sb.z};
  const R fb = vd3(tau, sb);
  const R t2b = R(-0.5) * f * f * fb;
  taub.x += R(2) * t2b * tau.x;
  taub.y += R(2) * t2b * tau.y;
  taub.z += R(2) * t2b * tau.z;
  // vp = vm + vm x tau
  const Vec<R> a1 = vx3(tau, vpb), a2 = vx3(vpb, vm);
  vmb = {vmb.x + vpb.x + a1.x, vmb.y + vpb.y + a1.y, vmb.z + vpb.z + a1.z};
  taub = {taub.x + a2.x, taub.y + a2.y, taub.z + a2.z};
  // tau = kq B ; vm = v + kq E
  const Vec<R> Bb = {kq * taub.x, kq * taub.y, kq * taub.z};
  Eb = {Eb.x + kq * vmb.x, Eb.y + kq * vmb.y, Eb.z + kq * vmb.z};
  // E = E0 + d x W ; B = B0 + beta d
  const Vec<R> Wb = vx3(Eb, d);
  const Vec<R> db1 = vx3(W, Eb);
  const R betab = vd3(Bb, d);
  A.rbx[p] = (rbx + dga[0]) + widen(db1.x + beta * Bb.x);
  A.rby[p] = (rby + dga[1]) + widen(db1.y + beta * Bb.y);
  A.rbz[p] = (rbz + dga[2]) + widen(db1.z + beta * Bb.z);
  vbx[p] = vmb.x;
  vby[p] = vmb.y;
  vbz[p] = vmb.z;
  out[0] = Eb.x; out[1] = Eb.y; out[2] = Eb.z;
  out[3] = Wb.x; out[4] = Wb.y; out[5] = Wb.z;
  out[6] = Bb.x; out[7] = Bb.y; out[8] = Bb.z;
  out[9] = betab;
}

template <typename R, bool DEP>
__global__ void __launch_bounds__(kThreads) k_push_adjoint(AdjArgs A) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  R g[10];
#pragma unroll
  for (int i = 0; i < 10; i++) g[i] = R(0);
  int32_t key = -1 - lane;
  if (p < A.n) {
    const int32_t T = A.tet[p];
    if (T >= 0 && T < A.nt) {
      const uint8_t s1 = A.status1[p];
      if (s1 != FEMPIC_P_OK) {   // frozen during the step: its later state does not enter the loss
        A.rbx[p] = A.rby[p] = A.rbz[p] = 0.0;
        static_cast<R*>(A.vbx)[p] = static_cast<R*>(A.vby)[p] = static_cast<R*>(A.vbz)[p] = R(0);
      }
      // ... but the charge it moved before it froze does
      if (s1 == FEMPIC_P_OK || (DEP && (s1 == FEMPIC_P_CAP || s1 == FEMPIC_P_ABSORBED))) {
        adjoint_particle<R, DEP>(A, p, T, g);
        key = T;
      }
    }
  }
  const unsigned full = 0xffffffffu;
  const int32_t prev = __shfl_up_sync(full, key, 1);
  const bool head = lane == 0 || prev != key;
  const unsigned heads = __ballot_sync(full, head);
  if (sizeof(R) == 4 && __popc(heads) > 4) {   // short runs: per-lane vector atomics
    if (key >= 0) {
      float* row = A.tetgrad32 + 12 * (int64_t)key;
      atomicAdd(reinterpret_cast<float4*>(row), make_float4((float)g[0], (float)g[1], (float)g[2], (float)g[3]));
      atomicAdd(reinterpret_cast<float4*>(row + 4), make_float4((float)g[4], (float)g[5], (float)g[6], (float)g[7]));
      atomicAdd(reinterpret_cast<float2*>(row + 8), make_float2((float)g[8], (float)g[9]));
    }
    return;
  }
  const unsigned above = lane == 31 ? 0u : (heads & (~0u << (lane + 1)));
  const int run_end = above ? (__ffs(above) - 2) : 31;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
    for (int i = 0; i < 10; i++) {
      const R o = __shfl_down_sync(full, g[i], off);
      if (lane + off <= run_end) g[i] += o;
    }
  }
  if (head && key >= 0) {
    if (sizeof(R) == 4) {   // mixed form: the run's sums into the tet's FP32 row
      float* row = A.tetgrad32 + 12 * (int64_t)key;
      atomicAdd(reinterpret_cast<float4*>(row), make_float4((float)g[0], (float)g[1], (float)g[2], (float)g[3]));
      atomicAdd(reinterpret_cast<float4*>(row + 4), make_float4((float)g[4], (float)g[5], (float)g[6], (float)g[7]));
      atomicAdd(reinterpret_cast<float2*>(row + 8), make_float2((float)g[8], (float)g[9]));
    } else {
      double* tg = A.tetgrad + 10 * (int64_t)key;
#pragma unroll
      for (int i = 0; i < 10; i++)
        if (g[i] != R(0)) atomicAdd(tg + i, (double)g[i]);
    }
  }
}

// Per-tet weights of the deposited-current loss L = sum_e u_e dG_e: alpha =
// sum_j u_{0j} G_j and beta = sum_{i<j} u_{ij} (G_i x G_j), with G_0 = -(G_1 +
// G_2 + G_3), so that a piece p -> q in the tet adds alpha . (q - p) + beta .
// ((p - x0) x (q - p)) to L per unit charge.
__global__ void __launch_bounds__(kThreads) k_current_weights(int64_t nt, const double* __restrict__ geom64,
                                                               const int4* __restrict__ te,
                                                               const double* __restrict__ u,
                                                               double* __restrict__ curw, int64_t ne,
                                                               unsigned long long* stats) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double G[4][3];
  grads64(geom64, (int32_t)t, G);
  const int4 e0 = te[2 * t], e1 = te[2 * t + 1];
  const int32_t eid[6] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y};
  double al[3] = {0.0, 0.0, 0.0}, be[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int e = 0; e < 6; e++) {
    const int i = le0(e), j = le1(e);
    const double ue = idx_in(eid[e], ne, stats) ? u[eid[e]] : 0.0;
    double c[3];
    cross3d(G[i], G[j], c);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      be[k] = fma(ue, c[k], be[k]);
      if (i == 0) al[k] = fma(ue, G[j][k], al[k]);
    }
  }
  double* o = curw + 6 * t;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    o[k] = al[k];
    o[3 + k] = be[k];
  }
}

// Transpose of the per-tet pre-pass for one step, first half: from the
// adjoint of (E0, W, B0, beta) to the adjoint of the carrier-restored DoFs
// eps (6 edges) and bet (4 faces) of each tet, written to tadj [nt][10]
// (zeros for a tet without particles).  The mixed form does it in FP32 from
// the FP32 tet record, the FP64 form in FP64.  The per-tet accumulators are
// cleared for the next step.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_field_adjoint(int64_t nt, const double* __restrict__ geom64,
                                                             const float4* __restrict__ rec,
                                                             double* __restrict__ tetgrad, float* __restrict__ tetgrad32,
                                                             double* __restrict__ tadj) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const bool mixed = sizeof(R) == 4;
  R a[10];
  bool any = false;
  if (!mixed) {
    double* tg = tetgrad + 10 * t;
#pragma unroll
    for (int i = 0; i < 10; i++) {
      const double v = tg[i];
      a[i] = (R)v;
      any = any || v != 0.0;
    }
    if (any) {
#pragma unroll
      for (int i = 0; i < 10; i++) tg[i] = 0.0;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 10; i++) a[i] = R(0);
  }
  if (mixed) {
    float4* r4 = reinterpret_cast<float4*>(tetgrad32 + 12 * t);
    const float4 u = r4[0], v = r4[1], w = r4[2];
    const float f[10] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w, w.x, w.y};
    bool any32 = false;
#pragma unroll
    for (int i = 0; i < 10; i++) {
      a[i] += (R)f[i];
      any32 = any32 || f[i] != 0.0f;
    }
    if (any32) {
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      r4[0] = z;
      r4[1] = z;
      r4[2] = z;
    }
    any = any || any32;
  }
  double* o = tadj + 10 * t;
  if (!any) {
#pragma unroll
    for (int i = 0; i < 10; i++) o[i] = 0.0;
    return;
  }
  V3<R> g[4];
  if (mixed) {
    const float4 q = rec[8 * t + 1], r = rec[8 * t + 2], c = rec[8 * t + 3];
    g[1] = {(R)q.z, (R)q.w, (R)r.x};
    g[2] = {(R)r.y, (R)r.z, (R)r.w};
    g[3] = {(R)c.x, (R)c.y, (R)c.z};
  } else {
    const double* G = geom64 + 12 * t;
    g[1] = {(R)G[3], (R)G[4], (R)G[5]};
    g[2] = {(R)G[6], (R)G[7], (R)G[8]};
    g[3] = {(R)G[9], (R)G[10], (R)G[11]};
  }
  // g_0 formed as in the forward pre-pass
  g[0] = {-(g[1].x + g[2].x + g[3].x), -(g[1].y + g[2].y + g[3].y), -(g[1].z + g[2].z + g[3].z)};
  const V3<R> E0b = {a[0], a[1], a[2]}, Wb = {a[3], a[4], a[5]}, B0b = {a[6], a[7], a[8]};
  const R betab = a[9];
  R epsb[6], betb[4];
#pragma unroll
  for (int e = 0; e < 6; e++) epsb[e] = vdot(Wb, vcross(g[le1(e)], g[le0(e)]));
  epsb[0] += vdot(E0b, g[1]);
  epsb[1] += vdot(E0b, g[2]);
  epsb[2] += vdot(E0b, g[3]);
  betb[0] = R(0);
  betb[1] = R(2) * vdot(B0b, vcross(g[2], g[3]));
  betb[2] = R(2) * vdot(B0b, vcross(g[1], g[3]));
  betb[3] = R(2) * vdot(B0b, vcross(g[1], g[2]));
#pragma unroll
  for (int f = 0; f < 4; f++) betb[f] += R(2) * betab * vdot(g[lf(f, 0)], vcross(g[lf(f, 1)], g[lf(f, 2)]));
#pragma unroll
  for (int e = 0; e < 6; e++) o[e] = widen(epsb[e]);
#pragma unroll
  for (int f = 0; f < 4; f++) o[6 + f] = widen(betb[f]);
}

// Second half: each edge and each face gathers its tets' terms (adjacency
// built once on the host: edge -> (tet, local edge), face -> (tet, local
// face)) and adds dL/dRe + j dL/dIm through eps = c_re Re(e~) - c_im Im(e~):
// one thread per edge or face, no atomics, a fixed summation order.
__global__ void __launch_bounds__(kThreads) k_dof_grad(int64_t ne, int64_t nf, const int32_t* __restrict__ estart,
                                                       const int32_t* __restrict__ eslot,
                                                       const int32_t* __restrict__ fslot,
                                                       const double* __restrict__ tadj, double cre, double cim,
                                                       double* __restrict__ egrad, double* __restrict__ bgrad,
                                                       int64_t nt, unsigned long long* stats) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < ne) {
    double sum = 0.0;
    for (int32_t j = estart[i]; j < estart[i + 1]; j++) {
      const int32_t sl = eslot[j];
      if (idx_in(sl, 6 * nt, stats)) sum += tadj[(int64_t)(sl / 6) * 10 + sl % 6];
    }
    if (sum != 0.0) {
      egrad[2 * i] += cre * sum;
      egrad[2 * i + 1] += -cim * sum;
    }
  }
  if (i < nf) {
    double sum = 0.0;
#pragma unroll
    for (int k = 0; k < 2; k++) {
      const int32_t sl = fslot[2 * i + k];
      if (sl >= 0 && idx_in(sl, 4 * nt, stats)) sum += tadj[(int64_t)(sl >> 2) * 10 + 6 + (sl & 3)];
    }
    if (sum != 0.0) {
      bgrad[2 * i] += cre * sum;
      bgrad[2 * i + 1] += -cim * sum;
    }
  }
}

// Total kinetic energy sum_p 1/2 m w |v|^2 over particles with tet >= 0 into
// *ke (FP64 atomics), and optionally the adjoint seed vbar = m w v, rbar = 0.
struct KEArgs {
  int64_t n;
  const void* vx;
  const void* vy;
  const void* vz;
  const int32_t* tet;
  Species sp;                // species ranges
  double mw[kMaxSpecies];    // m w per species
  double* ke;
  double* rbx;
  double* rby;
  double* rbz;
  void* vbx;
  void* vby;
  void* vbz;
};

template <typename R>
__global__ void __launch_bounds__(kThreads) k_kinetic_energy(KEArgs A) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t n = A.n;
  const void *vx = A.vx, *vy = A.vy, *vz = A.vz;
  void *vbx = A.vbx, *vby = A.vby, *vbz = A.vbz;
  double *rbx = A.rbx, *rby = A.rby, *rbz = A.rbz;
  double e = 0.0;
  if (p < n && A.tet[p] >= 0) {
    const double mw = A.mw[species_of(A.sp, p)];
    const double a = static_cast<const R*>(vx)[p], b = static_cast<const R*>(vy)[p], c = static_cast<const R*>(vz)[p];
    e = 0.5 * mw * (a * a + b * b + c * c);
    if (vbx) {
      static_cast<R*>(vbx)[p] = (R)(mw * a);
      static_cast<R*>(vby)[p] = (R)(mw * b);
      static_cast<R*>(vbz)[p] = (R)(mw * c);
      rbx[p] = rby[p] = rbz[p] = 0.0;
    }
  } else if (p < n && vbx) {
    static_cast<R*>(vbx)[p] = static_cast<R*>(vby)[p] = static_cast<R*>(vbz)[p] = R(0);
    rbx[p] = rby[p] = rbz[p] = 0.0;
  }
  for (int off = 16; off > 0; off >>= 1) e += __shfl_down_sync(0xffffffffu, e, off);
  if ((threadIdx.x & 31) == 0 && e != 0.0) atomicAdd(A.ke, e);
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T) + 16);
}

}  // namespace

// =================================================================== ABI
struct fempic_env {
  int device = 0;
  fempic_options opt{};
  HostMesh h;
  double* geom64 = nullptr;
  float4* tetrec = nullptr;
  int4* tn = nullptr;
  int4* nb = nullptr;
  int4* te = nullptr;
  int4* tf = nullptr;
  void* field = nullptr;
  double* dG = nullptr;
  unsigned long long* dGq = nullptr;   // 24-bit form [dGq_species][nt][8]
  int32_t dGq_species = 0;
  float4* tetdf = nullptr;             // contract form: low parts of grad lambda_1..3, [nt][4]
  double* mom = nullptr;               // contract form: moment slots [dGq_species][nt][6]
  float* momlo = nullptr;              // their low FP32 parts [dGq_species][nt][8]
  float4* tetout = nullptr;            // contract form: per-tet edge values of a step [nt][3]
  double* Gcum = nullptr;
  unsigned long long* stats = nullptr;
  int64_t* gstart = nullptr;
  int32_t* gtet = nullptr;
  double qw_last[kMaxSpecies] = {0};
  int32_t ns_last = 0;
  double* tetgrad = nullptr;        // adjoint of the per-tet affine field [nt][10]
  float* tetgrad32 = nullptr;       // mixed form: the same from per-lane atomics, [nt][12]
  double* tadj = nullptr;           // per-tet DoF-adjoint terms of one adjoint step [nt][10]
  double* curw = nullptr;           // deposited-current loss weights alpha, beta per tet [nt][6]
  bool curw_on = false;
  int32_t* estart = nullptr;        // edge -> (tet, local edge) slots, CSR [ne + 1]
  int32_t* eslot = nullptr;         // [6 nt], slot = 6 tet + local edge
  int32_t* fslot = nullptr;         // face -> (tet, local face) slots [nf][2], 4 tet + local face or -1
  CrossRec* xrec = nullptr;         // mixed form crossing queue [xtiles * 256]
  CrossRec64* xrec64 = nullptr;     // FP64 form crossing queue [xtiles * 256]
  int32_t* xcount = nullptr;        // [xtiles]
  int64_t xtiles = 0;
  int num_sms = 1;
  int tma_blocks_per_sm[2] = {0, 0}; // resident CTAs of the staged kernels (contract, 24-bit)
  int cross_blocks_per_sm[3] = {0, 0, 0};   // resident CTAs of the mixed crossing passes (-, contract, 24-bit)
  int64_t steps = 0;
  // per-kernel event timing (measurement support)
  struct Rec {
    int kid;
    int kernels;   // kernels launched inside the bracket
    cudaEvent_t a, b;
  };
  int32_t* sort_counts = nullptr;   // [sort_cap] per-key counters, then cursors
  int32_t* sort_offsets = nullptr;  // [sort_cap]
  bool deposit_on = true;           // fempic_set_deposit
  int32_t* sort_sums = nullptr;     // [sort_cap / 2048 + 1]
  int64_t sort_cap = 0;
  bool profiling = false;
  int32_t stall_cta = -1;           // fempic_debug_stall (test support)
  unsigned long long stall_ns = 0;
  unsigned long long seen_frozen = 0, seen_timeouts = 0, seen_bounds = 0;   // fempic_error_count baselines
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t pool_used = 0;
};

namespace {
constexpr size_t kMaxRecords = 65536;

// Brackets one kernel launch with events when profiling is on.
struct LaunchTimer {
  fempic_env* e;
  cudaStream_t st;
  int kid;
  int kernels = 0;   // kernels launched inside this bracket (not counting nested brackets)
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEvent_t take() {
    if (e->pool_used == e->pool.size()) {
      cudaEvent_t ev;
      if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
      e->pool.push_back(ev);
    }
    return e->pool[e->pool_used++];
  }
  LaunchTimer(fempic_env* env, cudaStream_t s, int k) : e(env), st(s), kid(k) {
    if (!e->profiling || e->recs.size() >= kMaxRecords) return;
    a = take();
    b = take();
    if (a && b) cudaEventRecord(a, st);
  }
  ~LaunchTimer() {
    if (a && b) {
      cudaEventRecord(b, st);
      e->recs.push_back({kid, kernels, a, b});
    }
  }
};
}  // namespace

static void free_env(fempic_env* e) {
  if (!e) return;
  for (cudaEvent_t ev : e->pool) cudaEventDestroy(ev);
  void* ptrs[] = {e->geom64, e->tetrec, e->tn, e->nb, e->te, e->tf, e->field, e->dG, e->dGq, e->tetdf, e->mom,
                  e->momlo, e->tetout,
                  e->Gcum, e->stats, e->gstart, e->gtet, e->sort_counts, e->sort_offsets, e->sort_sums, e->tetgrad, e->tetgrad32, e->tadj, e->curw, e->estart, e->eslot, e->fslot, e->xrec, e->xrec64, e->xcount,
                  nullptr};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete e;
}

extern "C" const char* fempic_last_error(void) { return g_last_error.c_str(); }

extern "C" void fempic_env_destroy(fempic_env* env) { free_env(env); }

static int upload(fempic_env* e) {
  const HostMesh& m = e->h;
  const int64_t nt = m.nt;
  std::vector<float4> geo(8 * nt), gdf(4 * nt);
  std::vector<int4> tn(nt), nb(nt), te(2 * nt), tf(nt);
  double max_coord = 0.0;
  for (int64_t i = 0; i < m.nn * 3; i++) max_coord = std::max(max_coord, std::fabs(m.xyz[i]));
  for (int64_t t = 0; t < nt; t++) {
    const double* G = &m.geom[12 * t];
    // mixed-form record: x0 exactly (3 x f64), FP32 gradients, the error
    // bound kappa of the FP32 inside test; the low FP32 parts of the
    // gradients go to tetdf (contract form)
    float g[9], glo[9];
    for (int i = 0; i < 9; i++) {
      g[i] = (float)G[3 + i];
      glo[i] = (float)(G[3 + i] - (double)g[i]);
    }
    // kappa bounds |FP32 lambda(b) - lambda(b)| for a segment start in the
    // tet: FP32 roundings of d, d + D, the gradients and the three-term
    // sums (each 2^-24 relative), amplified by |grad lambda_k|_1 and the
    // coordinate extent of the tet, plus the FP64 rounding of b.
    double gsum = 0.0, ext = 0.0;
    for (int k = 0; k < 4; k++) {
      double s1 = 0.0;
      for (int j = 0; j < 3; j++) {
        const double gk = k == 0 ? -(G[3 + j] + G[6 + j] + G[9 + j]) : G[3 * k + j];
        s1 += std::fabs(gk);
      }
      gsum = std::max(gsum, s1);
    }
    for (int i = 0; i < 4; i++)
      for (int j = 0; j < 4; j++)
        for (int a = 0; a < 3; a++)
          ext = std::max(ext, std::fabs(m.xyz[3 * (int64_t)m.tn[4 * t + i] + a] - m.xyz[3 * (int64_t)m.tn[4 * t + j] + a]));
    float kappa = (float)(0x1p-16 * (1.0 + 4.0 * gsum * ext) + gsum * max_coord * 0x1p-50);
    if (!(gsum * ext < 0x1p16)) kappa = INFINITY;   // a sliver: every particle takes the crossing pass
    float head[16];
    std::memcpy(head, G, 24);   // x0 as 6 words, bits unchanged
    std::memcpy(head + 6, g, sizeof(g));
    head[15] = kappa;
    std::memcpy(&geo[8 * t], head, sizeof(head));
    for (int k = 4; k < 7; k++) geo[8 * t + k] = make_float4(0.f, 0.f, 0.f, 0.f);
    gdf[4 * t] = make_float4(glo[0], glo[1], glo[2], glo[3]);
    gdf[4 * t + 1] = make_float4(glo[4], glo[5], glo[6], glo[7]);
    gdf[4 * t + 2] = make_float4(glo[8], 0.f, 0.f, 0.f);
    gdf[4 * t + 3] = make_float4(0.f, 0.f, 0.f, 0.f);
    {
      // face maps of the mixed crossing walk, 16 bits per local face k with a
      // neighbour: bits 0-1 the neighbour's local node that is not in this
      // tet (its entry face), bits 2+2i the local node of this tet that is
      // the neighbour's local node i (any value for the entry node)
      uint32_t fmap[2] = {0u, 0u};
      for (int k = 0; k < 4; k++) {
        const int32_t nbt = m.nb[4 * t + k];
        if (nbt < 0) continue;
        uint32_t code = 0u;
        for (int i2 = 0; i2 < 4; i2++) {
          int hit = -1;
          for (int j = 0; j < 4; j++)
            if (m.tn[4 * t + j] == m.tn[4 * (int64_t)nbt + i2]) hit = j;
          if (hit < 0)
            code |= (uint32_t)i2;
          else
            code |= (uint32_t)hit << (2 + 2 * i2);
        }
        fmap[k >> 1] |= code << (16 * (k & 1));
      }
      std::memcpy(&geo[8 * t + 6].z, &fmap[0], 4);
      std::memcpy(&geo[8 * t + 6].w, &fmap[1], 4);
    }
    int32_t nbk[4] = {m.nb[4 * t], m.nb[4 * t + 1], m.nb[4 * t + 2], m.nb[4 * t + 3]};
    float4 nbf;
    std::memcpy(&nbf, nbk, sizeof(nbf));
    geo[8 * t + 7] = nbf;
    tn[t] = make_int4(m.tn[4 * t], m.tn[4 * t + 1], m.tn[4 * t + 2], m.tn[4 * t + 3]);
    nb[t] = make_int4(m.nb[4 * t], m.nb[4 * t + 1], m.nb[4 * t + 2], m.nb[4 * t + 3]);
    te[2 * t] = make_int4(m.te[6 * t], m.te[6 * t + 1], m.te[6 * t + 2], m.te[6 * t + 3]);
    te[2 * t + 1] = make_int4(m.te[6 * t + 4], m.te[6 * t + 5], 0, 0);
    tf[t] = make_int4(m.tf[4 * t], m.tf[4 * t + 1], m.tf[4 * t + 2], m.tf[4 * t + 3]);
  }
  FEMPIC_CUDA(dalloc(&e->geom64, 12 * nt));
  FEMPIC_CUDA(dalloc(&e->tetrec, 8 * nt));
  FEMPIC_CUDA(dalloc(&e->tn, nt));
  FEMPIC_CUDA(dalloc(&e->nb, nt));
  FEMPIC_CUDA(dalloc(&e->te, 2 * nt));
  FEMPIC_CUDA(dalloc(&e->tf, nt));
  FEMPIC_CUDA(cudaMemcpy(e->geom64, m.geom.data(), 12 * nt * sizeof(double), cudaMemcpyHostToDevice));
  FEMPIC_CUDA(cudaMemcpy(e->tetrec, geo.data(), 8 * nt * sizeof(float4), cudaMemcpyHostToDevice));
  if (e->opt.precision == FEMPIC_MIXED) {
    FEMPIC_CUDA(dalloc(&e->tetdf, 4 * nt));
    FEMPIC_CUDA(cudaMemcpy(e->tetdf, gdf.data(), 4 * nt * sizeof(float4), cudaMemcpyHostToDevice));
  }
  FEMPIC_CUDA(cudaMemcpy(e->tn, tn.data(), nt * sizeof(int4), cudaMemcpyHostToDevice));
  FEMPIC_CUDA(cudaMemcpy(e->nb, nb.data(), nt * sizeof(int4), cudaMemcpyHostToDevice));
  FEMPIC_CUDA(cudaMemcpy(e->te, te.data(), 2 * nt * sizeof(int4), cudaMemcpyHostToDevice));
  FEMPIC_CUDA(cudaMemcpy(e->tf, tf.data(), nt * sizeof(int4), cudaMemcpyHostToDevice));
  {
    // adjacency of the adjoint's DoF-gradient gathers
    std::vector<int32_t> estart(m.ne + 1, 0), eslot(6 * nt), fslot(2 * m.nf, -1);
    for (int64_t i = 0; i < 6 * nt; i++) estart[m.te[i] + 1]++;
    for (int64_t k = 0; k < m.ne; k++) estart[k + 1] += estart[k];
    std::vector<int32_t> cur(estart.begin(), estart.end() - 1);
    for (int64_t i = 0; i < 6 * nt; i++) eslot[cur[m.te[i]]++] = (int32_t)i;
    for (int64_t i = 0; i < 4 * nt; i++) {
      const int32_t f = m.tf[i];
      if (fslot[2 * f] < 0)
        fslot[2 * f] = (int32_t)i;
      else
        fslot[2 * f + 1] = (int32_t)i;
    }
    FEMPIC_CUDA(dalloc(&e->estart, m.ne + 1));
    FEMPIC_CUDA(dalloc(&e->eslot, 6 * nt));
    FEMPIC_CUDA(dalloc(&e->fslot, 2 * m.nf));
    FEMPIC_CUDA(cudaMemcpy(e->estart, estart.data(), (m.ne + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    FEMPIC_CUDA(cudaMemcpy(e->eslot, eslot.data(), 6 * nt * sizeof(int32_t), cudaMemcpyHostToDevice));
    FEMPIC_CUDA(cudaMemcpy(e->fslot, fslot.data(), 2 * m.nf * sizeof(int32_t), cudaMemcpyHostToDevice));
  }
  if (e->opt.precision == FEMPIC_FP64) {
    FEMPIC_CUDA(dalloc(reinterpret_cast<double**>(&e->field), 10 * nt));
    FEMPIC_CUDA(dalloc(&e->dG, m.ne));
    FEMPIC_CUDA(cudaMemset(e->dG, 0, m.ne * sizeof(double)));
  }
  FEMPIC_CUDA(dalloc(&e->Gcum, m.ne));
  FEMPIC_CUDA(cudaMemset(e->Gcum, 0, m.ne * sizeof(double)));
  FEMPIC_CUDA(dalloc(&e->stats, 4));
  FEMPIC_CUDA(cudaMemset(e->stats, 0, 4 * sizeof(unsigned long long)));
  FEMPIC_CUDA(dalloc(&e->gstart, m.gstart.size()));
  FEMPIC_CUDA(dalloc(&e->gtet, m.gtet.size() + 1));
  FEMPIC_CUDA(cudaMemcpy(e->gstart, m.gstart.data(), m.gstart.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  if (!m.gtet.empty())
    FEMPIC_CUDA(cudaMemcpy(e->gtet, m.gtet.data(), m.gtet.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  FEMPIC_CUDA(cudaDeviceSynchronize());
  return FEMPIC_OK;
}

extern "C" int fempic_env_create(const fempic_mesh_desc* mesh, const fempic_options* opts, fempic_env** out) {
  g_last_error.clear();
  if (!mesh || !opts || !out) return fail(FEMPIC_EINVAL, "env_create: NULL argument");
  *out = nullptr;
  if ((opts->precision != FEMPIC_FP64 && opts->precision != FEMPIC_MIXED && opts->precision != FEMPIC_MIXED_Q24) ||
      opts->max_crossings < 0 ||
      opts->max_crossings > kMaxCrossingsLimit ||
      (opts->wall_mode != FEMPIC_WALL_REFLECT && opts->wall_mode != FEMPIC_WALL_ABSORB) || opts->reserved != 0)
    return fail(FEMPIC_EINVAL, "env_create: bad options");
  fempic_env* e = new (std::nothrow) fempic_env();
  if (!e) return fail(FEMPIC_ENOMEM, "env_create: host allocation");
  e->opt = *opts;
  if (cudaGetDevice(&e->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&e->num_sms, cudaDevAttrMultiProcessorCount, e->device) != cudaSuccess) {
    delete e;
    return fail(FEMPIC_ECUDA, "env_create: no CUDA device");
  }
  std::string err;
  int rc = build_host_mesh(*mesh, &e->h, &err);
  if (rc != FEMPIC_OK) {
    delete e;
    return fail(rc, err);
  }
  rc = upload(e);
  if (rc != FEMPIC_OK) {
    free_env(e);
    return rc;
  }
  *out = e;
  return FEMPIC_OK;
}

extern "C" int fempic_env_query(const fempic_env* env, int64_t* counts4, int32_t* tet_nodes, int32_t* edge_nodes,
                                int32_t* face_nodes, int32_t* tet_edges, int32_t* tet_faces, int32_t* tet_nbr) {
  if (!env) return fail(FEMPIC_EINVAL, "env_query: NULL env");
  const HostMesh& m = env->h;
  if (counts4) {
    counts4[0] = m.nn;
    counts4[1] = m.ne;
    counts4[2] = m.nf;
    counts4[3] = m.nt;
  }
  if (tet_nodes) std::memcpy(tet_nodes, m.tn.data(), m.tn.size() * sizeof(int32_t));
  if (edge_nodes) std::memcpy(edge_nodes, m.en.data(), m.en.size() * sizeof(int32_t));
  if (face_nodes) std::memcpy(face_nodes, m.fn.data(), m.fn.size() * sizeof(int32_t));
  if (tet_edges) std::memcpy(tet_edges, m.te.data(), m.te.size() * sizeof(int32_t));
  if (tet_faces) std::memcpy(tet_faces, m.tf.data(), m.tf.size() * sizeof(int32_t));
  if (tet_nbr) std::memcpy(tet_nbr, m.nb.data(), m.nb.size() * sizeof(int32_t));
  return FEMPIC_OK;
}

static int check_particles(const fempic_particles* p, bool need_v) {
  if (!p) return fail(FEMPIC_EINVAL, "particles: NULL");
  if (p->n < 0) return fail(FEMPIC_EINVAL, "particles: negative count");
  if (p->n == 0) return FEMPIC_OK;
  if (!p->x || !p->y || !p->z || !p->tet || !p->status)
    return fail(FEMPIC_EINVAL, "particles: NULL position/tet/status array");
  if (need_v && (!p->vx || !p->vy || !p->vz)) return fail(FEMPIC_EINVAL, "particles: NULL velocity array");
  return FEMPIC_OK;
}

static int fill_species(const fempic_particles* p, double dt, Species* sp) {
  if (p->n_species < 1 || p->n_species > kMaxSpecies || !p->species_begin || !p->q || !p->m || !p->w)
    return fail(FEMPIC_EINVAL, "particles: species table (1..8 ranges, q, m, w)");
  sp->ns = p->n_species;
  if (p->species_begin[0] != 0 || p->species_begin[p->n_species] != p->n)
    return fail(FEMPIC_EINVAL, "particles: species ranges must cover [0, n)");
  for (int s = 0; s <= p->n_species; s++) {
    sp->begin[s] = p->species_begin[s];
    if (s > 0 && sp->begin[s] < sp->begin[s - 1]) return fail(FEMPIC_EINVAL, "particles: species ranges decrease");
  }
  for (int s = p->n_species + 1; s <= kMaxSpecies; s++) sp->begin[s] = p->n;
  for (int s = 0; s < p->n_species; s++) {
    if (!(p->m[s] > 0.0)) return fail(FEMPIC_EINVAL, "particles: mass must be > 0");
    sp->kq[s] = ((p->q[s] / p->m[s]) * dt) * 0.5;
    sp->qw[s] = p->q[s] * p->w[s];
    sp->kq32[s] = (float)sp->kq[s];
  }
  for (int s = p->n_species; s < kMaxSpecies; s++) {
    sp->kq[s] = sp->qw[s] = 0.0;
    sp->kq32[s] = 0.f;
  }
  return FEMPIC_OK;
}

static unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

extern "C" int fempic_locate(fempic_env* env, const fempic_particles* p, void* stream) {
  if (!env) return fail(FEMPIC_EINVAL, "locate: NULL env");
  int rc = check_particles(p, false);
  if (rc) return rc;
  if (p->n == 0) return FEMPIC_OK;
  LocateArgs A{};
  A.n = p->n;
  A.x = p->x;
  A.y = p->y;
  A.z = p->z;
  A.tet = p->tet;
  A.status = p->status;
  A.geom64 = env->geom64;
  A.gstart = env->gstart;
  A.gtet = env->gtet;
  A.nt = env->h.nt;
  A.stats = env->stats;
  for (int a = 0; a < 3; a++) {
    A.gd[a] = env->h.gd[a];
    A.ginv[a] = env->h.ginv[a];
    A.lo[a] = env->h.lo[a];
  }
  {
    LaunchTimer lt(env, (cudaStream_t)stream, FEMPIC_K_LOCATE);
    k_locate<<<blocks_for(p->n), kThreads, 0, (cudaStream_t)stream>>>(A);
    lt.kernels = 1;
  }
  FEMPIC_CUDA(cudaGetLastError());
  return FEMPIC_OK;
}

// Crossing queue of the mixed form: a 256-record region per tile of 256
// particles plus a count per tile, grown on demand (every tile count is
// rewritten by the common path each step, so nothing needs clearing).
static int ensure_xqueue(fempic_env* env, int64_t n, cudaStream_t st) {
  const int64_t tiles = (n + kThreads - 1) / kThreads;
  if (env->xtiles >= tiles) return FEMPIC_OK;
  if (env->xcount) {
    FEMPIC_CUDA(cudaStreamSynchronize(st));
    cudaFree(env->xrec);
    cudaFree(env->xrec64);
    cudaFree(env->xcount);
    env->xrec = nullptr;
    env->xrec64 = nullptr;
    env->xcount = nullptr;
    env->xtiles = 0;
  }
  if (env->opt.precision != FEMPIC_FP64)
    FEMPIC_CUDA(dalloc(&env->xrec, tiles * kThreads));
  else
    FEMPIC_CUDA(dalloc(&env->xrec64, tiles * kThreads));
  FEMPIC_CUDA(dalloc(&env->xcount, tiles));
  env->xtiles = tiles;
  return FEMPIC_OK;
}

static int ensure_mixed_accumulators(fempic_env* env, int ns, cudaStream_t st) {
  const bool q24 = env->opt.precision == FEMPIC_MIXED_Q24;
  if ((q24 ? env->dGq != nullptr : env->mom != nullptr) && env->dGq_species >= ns) return FEMPIC_OK;
  // The slots hold one step only; a larger species count reallocates them,
  // so a step must be finalized (fempic_deposit) before the species table
  // grows.
  const size_t nslot = (size_t)ns * env->h.nt * 8;
  if (env->dGq || env->mom) FEMPIC_CUDA(cudaStreamSynchronize(st));
  if (q24) {
    unsigned long long* nq = nullptr;
    FEMPIC_CUDA(dalloc(&nq, nslot));
    FEMPIC_CUDA(cudaMemsetAsync(nq, 0, nslot * sizeof(unsigned long long), st));
    if (env->dGq) cudaFree(env->dGq);
    env->dGq = nq;
  } else {
    const size_t nmom = (size_t)ns * env->h.nt * 6;
    double* nm = nullptr;
    float* nl = nullptr;
    FEMPIC_CUDA(dalloc(&nm, nmom));
    FEMPIC_CUDA(dalloc(&nl, nslot));
    FEMPIC_CUDA(cudaMemsetAsync(nm, 0, nmom * sizeof(double), st));
    FEMPIC_CUDA(cudaMemsetAsync(nl, 0, nslot * sizeof(float), st));
    if (env->mom) {
      cudaFree(env->mom);
      cudaFree(env->momlo);
    }
    env->mom = nm;
    env->momlo = nl;
    if (!env->tetout) {
      FEMPIC_CUDA(dalloc(&env->tetout, 3 * env->h.nt));
      FEMPIC_CUDA(cudaMemsetAsync(env->tetout, 0, 3 * env->h.nt * sizeof(float4), st));
    }
  }
  env->dGq_species = ns;
  return FEMPIC_OK;
}

// Host view of the envelope of one step: nl DoF levels with weights N_k(t).
struct HostLevels {
  int nl;
  const void* e[3];
  const void* b[3];
  double w[3];
  double amp;
};

// Every argument check of a push step, on the host, before any device work.
static int validate_step(const fempic_particles* p, const HostLevels& H, double omega0, double t, double dt,
                         Species* sp) {
  int rc = check_particles(p, true);
  if (rc) return rc;
  for (int k = 0; k < H.nl; k++)
    if (!H.e[k] || !H.b[k]) return fail(FEMPIC_EINVAL, "push_step: NULL DoF arrays");
  if (!(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(omega0) || !std::isfinite(t) || !std::isfinite(H.amp))
    return fail(FEMPIC_EINVAL, "push_step: non-finite or non-positive scalar");
  for (int k = 0; k < H.nl; k++)
    if (!std::isfinite(H.w[k])) return fail(FEMPIC_EINVAL, "push_step: non-finite level weight");
  return fill_species(p, dt, sp);
}

// Resident CTAs per SM of a mixed crossing pass (1 contract, 2 24-bit),
// cached per env: the passes hand records out along per-warp streams, so
// one wave of resident CTAs (no second partial wave) measured fastest
// (contract pass 0.200 -> 0.186 ms per step at 10M particles).
static int cross_resident(fempic_env* env, int which, int* out) {
  int& bps = env->cross_blocks_per_sm[which];
  if (bps == 0) {
    int nb = 0;
    if (which == 1)
      FEMPIC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cross_df, kThreads, 0));
    else
      FEMPIC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cross_q24, kThreads, 0));
    bps = nb > 0 ? nb : 1;
  }
  *out = bps;
  return FEMPIC_OK;
}

static int push_step_impl(fempic_env* env, const fempic_particles* p, const HostLevels& H, double omega0,
                          double t, double dt, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  PushArgs A{};
  int rc = validate_step(p, H, omega0, t, dt, &A.sp);
  if (rc) return rc;
  const bool mixed = env->opt.precision != FEMPIC_FP64;
  const bool q24 = env->opt.precision == FEMPIC_MIXED_Q24;
  if (mixed) {
    rc = ensure_mixed_accumulators(env, p->n_species, st);
    if (rc) return rc;
  }
  // (c) carrier: phase and c in FP64 on the host; level k enters with c N_k(t)
  const double phi = omega0 * t;
  const double cre = H.amp * std::cos(phi), cim = H.amp * std::sin(phi);
  const int64_t nt = env->h.nt;
  {
  LaunchTimer lt(env, st, FEMPIC_K_FIELD);
  lt.kernels = 1;
  if (mixed) {
    Levels<float2, float> L{};
    L.ne = env->h.ne;
    L.nf = env->h.nf;
    L.stats = env->stats;
    for (int k = 0; k < H.nl; k++) {
      L.e[k] = static_cast<const float2*>(H.e[k]);
      L.b[k] = static_cast<const float2*>(H.b[k]);
      L.cre[k] = (float)(cre * H.w[k]);
      L.cim[k] = (float)(cim * H.w[k]);
    }
    if (H.nl == 1)
      k_field_f32<1><<<blocks_for(nt), kThreads, 0, st>>>(nt, env->tetrec, env->te, env->tf, L);
    else
      k_field_f32<3><<<blocks_for(nt), kThreads, 0, st>>>(nt, env->tetrec, env->te, env->tf, L);
  } else {
    Levels<double2, double> L{};
    L.ne = env->h.ne;
    L.nf = env->h.nf;
    L.stats = env->stats;
    for (int k = 0; k < H.nl; k++) {
      L.e[k] = static_cast<const double2*>(H.e[k]);
      L.b[k] = static_cast<const double2*>(H.b[k]);
      L.cre[k] = cre * H.w[k];
      L.cim[k] = cim * H.w[k];
    }
    if (H.nl == 1)
      k_field_fp64<1><<<blocks_for(nt), kThreads, 0, st>>>(nt, env->geom64, env->te, env->tf, L,
                                                            static_cast<double*>(env->field));
    else
      k_field_fp64<3><<<blocks_for(nt), kThreads, 0, st>>>(nt, env->geom64, env->te, env->tf, L,
                                                            static_cast<double*>(env->field));
  }
  }
  FEMPIC_CUDA(cudaGetLastError());
  env->ns_last = p->n_species;
  for (int s = 0; s < kMaxSpecies; s++) env->qw_last[s] = A.sp.qw[s];
  env->steps++;
  if (p->n == 0) return FEMPIC_OK;
  A.n = p->n;
  A.x = p->x;
  A.y = p->y;
  A.z = p->z;
  A.vx = p->vx;
  A.vy = p->vy;
  A.vz = p->vz;
  A.tet = p->tet;
  A.status = p->status;
  A.ncross = p->n_cross;
  A.dt = dt;
  A.dt32 = (float)dt;
  A.max_cross = env->opt.max_crossings;
  A.wall_mode = env->opt.wall_mode;
  for (int a = 0; a < 3; a++) {
    A.lo[a] = env->h.lo[a];
    A.hi[a] = env->h.hi[a];
  }
  A.nt = nt;
  A.ne = env->h.ne;
  A.geom64 = env->geom64;
  A.tetrec = env->tetrec;
  A.tn = env->tn;
  A.nb = env->nb;
  A.te = env->te;
  A.field = env->field;
  A.dG = env->deposit_on ? env->dG : nullptr;
  A.dGq = env->deposit_on ? env->dGq : nullptr;
  A.mom = env->deposit_on ? env->mom : nullptr;
  A.momlo = env->momlo;
  A.tetdf = env->tetdf;
  A.stats = env->stats;
  rc = ensure_xqueue(env, p->n, st);
  if (rc) return rc;
  A.xrec = env->xrec;
  A.xrec64 = env->xrec64;
  A.xcount = env->xcount;
  A.wait_ns = env->stall_cta >= 0 ? env->stall_ns : kWaitLimitNs;
  A.stall_cta = env->stall_cta;
  env->stall_cta = -1;   // one launch only
  {
    LaunchTimer lt(env, st, FEMPIC_K_PUSH);
    if (mixed) {
      // bulk copies need 16-byte aligned sources: stage full tiles when every
      // particle array allows it; the ragged tail (or everything) goes plain
      const uintptr_t align = (uintptr_t)p->x | (uintptr_t)p->y | (uintptr_t)p->z | (uintptr_t)p->vx |
                              (uintptr_t)p->vy | (uintptr_t)p->vz | (uintptr_t)p->tet;
      const int64_t ntiles = (FEMPIC_USE_TMA && !(align & 15u)) ? p->n / kTile : 0;
      if (ntiles > 0) {
        int& bps = env->tma_blocks_per_sm[q24 ? 1 : 0];
        if (bps == 0) {
          int nb = 0;
          if (q24)
            FEMPIC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push_mixed_tma<true>, kThreads, 0));
          else
            FEMPIC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push_mixed_tma<false>, kThreads, 0));
          bps = nb > 0 ? nb : 1;
        }
        const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)env->num_sms * bps);
        if (q24)
          k_push_mixed_tma<true><<<grid, kThreads, 0, st>>>(A, ntiles);
        else
          k_push_mixed_tma<false><<<grid, kThreads, 0, st>>>(A, ntiles);
        lt.kernels++;
      }
      const int64_t rest = p->n - ntiles * kTile;
      if (rest > 0) {
        if (q24)
          k_push_mixed<true><<<blocks_for(rest), kThreads, 0, st>>>(A, ntiles * kTile);
        else
          k_push_mixed<false><<<blocks_for(rest), kThreads, 0, st>>>(A, ntiles * kTile);
        lt.kernels++;
      }
      const int64_t all_tiles = (p->n + kTile - 1) / kTile;
      int cb = 0;
      rc = cross_resident(env, q24 ? 2 : 1, &cb);
      if (rc) return rc;
      const unsigned cross_blocks = (unsigned)std::min<int64_t>((all_tiles + 7) / 8, (int64_t)env->num_sms * cb);
      LaunchTimer lc(env, st, FEMPIC_K_CROSS);   // nested: also inside the push bracket
      if (q24)
        k_cross_q24<<<cross_blocks, kThreads, 0, st>>>(A, all_tiles);
      else
        k_cross_df<<<cross_blocks, kThreads, 0, st>>>(A, all_tiles);
      lc.kernels = 1;
    } else {
      k_push_fp64<<<blocks_for(p->n), kThreads, 0, st>>>(A);
      lt.kernels = 1;
      // the FP64 walk is FP64-pipe bound: 8 CTAs per SM queued (about three
      // resident waves) measured faster than one resident wave
      const int64_t all_tiles = (p->n + kThreads - 1) / kThreads;
      const unsigned cross_blocks = (unsigned)std::min<int64_t>((all_tiles + 7) / 8, (int64_t)env->num_sms * 8);
      LaunchTimer lc(env, st, FEMPIC_K_CROSS);   // nested: also inside the push bracket
      k_cross_fp64<<<cross_blocks, kThreads, 0, st>>>(A, all_tiles);
      lc.kernels = 1;
    }
  }
  FEMPIC_CUDA(cudaGetLastError());
  return FEMPIC_OK;
}

extern "C" int fempic_push_step(fempic_env* env, const fempic_particles* p, const fempic_envelope* envl,
                                double omega0, double t, double dt, void* stream) {
  if (!env || !envl) return fail(FEMPIC_EINVAL, "push_step: NULL env/envelope");
  HostLevels H{};
  H.nl = 1;
  H.e[0] = envl->e_tilde;
  H.b[0] = envl->b_tilde;
  H.w[0] = 1.0;
  H.amp = envl->amp;
  return push_step_impl(env, p, H, omega0, t, dt, stream);
}

extern "C" int fempic_push_step3(fempic_env* env, const fempic_particles* p, const fempic_envelope3* envl,
                                 double omega0, double t, double dt, void* stream) {
  if (!env || !envl) return fail(FEMPIC_EINVAL, "push_step3: NULL env/envelope");
  HostLevels H{};
  H.nl = 3;
  for (int k = 0; k < 3; k++) {
    H.e[k] = envl->e_tilde[k];
    H.b[k] = envl->b_tilde[k];
    H.w[k] = envl->weight[k];
  }
  H.amp = envl->amp;
  return push_step_impl(env, p, H, omega0, t, dt, stream);
}

namespace fempic {
int env_precision(const fempic_env* env) { return env->opt.precision; }

unsigned long long* env_stats(fempic_env* env) { return env->stats; }

int validate_push_step(const fempic_particles* p, const fempic_envelope* envl, double omega0, double t,
                       double dt) {
  if (!envl) return fail(FEMPIC_EINVAL, "push_step: NULL envelope");
  HostLevels H{};
  H.nl = 1;
  H.e[0] = envl->e_tilde;
  H.b[0] = envl->b_tilde;
  H.w[0] = 1.0;
  H.amp = envl->amp;
  Species sp{};
  return validate_step(p, H, omega0, t, dt, &sp);
}
}  // namespace fempic

extern "C" int fempic_lagrange3(const double* tau, double t, double* w_out) {
  if (!tau || !w_out) return fail(FEMPIC_EINVAL, "lagrange3: NULL argument");
  if (!std::isfinite(t) || !std::isfinite(tau[0]) || !std::isfinite(tau[1]) || !std::isfinite(tau[2]) ||
      tau[0] == tau[1] || tau[1] == tau[2] || tau[0] == tau[2])
    return fail(FEMPIC_EINVAL, "lagrange3: level times must be finite and distinct");
  for (int k = 0; k < 3; k++) {
    double w = 1.0;
    for (int j = 0; j < 3; j++)
      if (j != k) w *= (t - tau[j]) / (tau[k] - tau[j]);
    w_out[k] = w;
  }
  return FEMPIC_OK;
}

static int deposit_impl(fempic_env* env, double omega0, double t_next, double* dG_out, double* G_cum_out,
                        void* G_env_out, bool local, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const int prec = env->opt.precision;
  FinalizeArgs A{};
  A.ne = env->h.ne;
  A.nt = env->h.nt;
  A.stats = env->stats;
  A.mode = prec == FEMPIC_FP64 ? 0 : (prec == FEMPIC_MIXED ? 1 : 2);
  A.ns = env->ns_last;
  for (int s = 0; s < kMaxSpecies; s++) A.qwscale[s] = env->qw_last[s] * 0x1p-48;
  A.dG = env->dG;
  A.dGq = env->dGq;
  A.tetout = reinterpret_cast<const float*>(env->tetout);
  A.Gcum = env->Gcum;
  A.dG_out = dG_out;
  A.Gcum_out = G_cum_out;
  A.Genv_out = static_cast<double2*>(G_env_out);
  A.estart = env->estart;
  A.eslot = env->eslot;
  A.local = local ? 1 : 0;
  const double phi = omega0 * t_next;
  A.c = std::cos(phi);
  A.s = std::sin(phi);
  if (A.mode == 2 && !env->dGq) A.ns = 0;
  if (A.mode == 1 && !env->mom) {
    int rc = ensure_mixed_accumulators(env, 1, st);   // no step yet: the pull reads zeros
    if (rc) return rc;
    A.tetout = reinterpret_cast<const float*>(env->tetout);
    A.ns = 0;
  }
  {
    LaunchTimer lt(env, st, FEMPIC_K_FINALIZE);
    if (A.mode == 1) {
      TetFinalizeArgs T{};
      T.nt = env->h.nt;
      T.ns = A.ns;
      T.tetrec = env->tetrec;
      T.tetdf = env->tetdf;
      T.mom = env->mom;
      T.momlo = env->momlo;
      for (int s = 0; s < kMaxSpecies; s++) {
        T.qwh[s] = (float)env->qw_last[s];
        T.qwl[s] = (float)(env->qw_last[s] - (double)T.qwh[s]);
      }
      T.out = env->tetout;
      k_tet_finalize<<<blocks_for(T.nt), kThreads, 0, st>>>(T);
      lt.kernels++;
    }
    k_deposit_finalize<<<blocks_for(A.ne), kThreads, 0, st>>>(A);
    lt.kernels++;
    if (A.mode == 2 && A.ns > 0)
      FEMPIC_CUDA(cudaMemsetAsync(env->dGq, 0, (size_t)A.ns * env->h.nt * 8 * sizeof(unsigned long long), st));
  }
  FEMPIC_CUDA(cudaGetLastError());
  return FEMPIC_OK;
}

extern "C" int fempic_deposit(fempic_env* env, double omega0, double t_next, double* dG_out, double* G_cum_out,
                              void* G_env_out, void* stream) {
  if (!env) return fail(FEMPIC_EINVAL, "deposit: NULL env");
  if (!std::isfinite(omega0) || !std::isfinite(t_next)) return fail(FEMPIC_EINVAL, "deposit: non-finite scalar");
  return deposit_impl(env, omega0, t_next, dG_out, G_cum_out, G_env_out, false, stream);
}

extern "C" int fempic_deposit_local(fempic_env* env, double* dG_out, void* stream) {
  if (!env || !dG_out) return fail(FEMPIC_EINVAL, "deposit_local: NULL env or dG_out");
  return deposit_impl(env, 0.0, 0.0, dG_out, nullptr, nullptr, true, stream);
}

extern "C" int fempic_accumulate(fempic_env* env, double omega0, double t_next, const double* dG, double* G_cum_out,
                                 void* G_env_out, void* stream) {
  if (!env || !dG) return fail(FEMPIC_EINVAL, "accumulate: NULL env or dG");
  if (!std::isfinite(omega0) || !std::isfinite(t_next)) return fail(FEMPIC_EINVAL, "accumulate: non-finite scalar");
  const double phi = omega0 * t_next;
  {
    LaunchTimer lt(env, (cudaStream_t)stream, FEMPIC_K_FINALIZE);
    k_accumulate<<<blocks_for(env->h.ne), kThreads, 0, (cudaStream_t)stream>>>(
        env->h.ne, dG, env->Gcum, G_cum_out, static_cast<double2*>(G_env_out), std::cos(phi), std::sin(phi));
    lt.kernels = 1;
  }
  FEMPIC_CUDA(cudaGetLastError());
  return FEMPIC_OK;
}

extern "C" int fempic_set_deposit(fempic_env* env, int32_t enable) {
  if (!env) return fail(FEMPIC_EINVAL, "set_deposit: NULL env");
  env->deposit_on = enable != 0;
  return FEMPIC_OK;
}

extern "C" int fempic_reset_deposit(fempic_env* env, void* stream) {
  if (!env) return fail(FEMPIC_EINVAL, "reset_deposit: NULL env");
  cudaStream_t st = (cudaStream_t)stream;
  FEMPIC_CUDA(cudaMemsetAsync(env->Gcum, 0, env->h.ne * sizeof(double), st));
  if (env->dG) FEMPIC_CUDA(cudaMemsetAsync(env->dG, 0, env->h.ne * sizeof(double), st));
  const size_t nslot = (size_t)env->dGq_species * env->h.nt * 8;
  if (env->dGq) FEMPIC_CUDA(cudaMemsetAsync(env->dGq, 0, nslot * sizeof(unsigned long long), st));
  if (env->mom) {
    FEMPIC_CUDA(cudaMemsetAsync(env->mom, 0, (size_t)env->dGq_species * env->h.nt * 6 * sizeof(double), st));
    FEMPIC_CUDA(cudaMemsetAsync(env->momlo, 0, nslot * sizeof(float), st));
  }
  return FEMPIC_OK;
}

extern "C" int fempic_nodal_charge(fempic_env* env, const fempic_particles* p, double* rho, void* stream) {
  if (!env || !rho) return fail(FEMPIC_EINVAL, "nodal_charge: NULL env/rho");
  int rc = check_particles(p, false);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  FEMPIC_CUDA(cudaMemsetAsync(rho, 0, env->h.nn * sizeof(double), st));
  if (p->n == 0) return FEMPIC_OK;
  ChargeArgs A{};
  rc = fill_species(p, 1.0, &A.sp);
  if (rc) return rc;
  A.n = p->n;
  A.x = p->x;
  A.y = p->y;
  A.z = p->z;
  A.tet = p->tet;
  A.nt = env->h.nt;
  A.q24 = env->opt.precision == FEMPIC_MIXED_Q24;
  A.geom64 = env->geom64;
  A.tetrec = env->tetrec;
  A.tn = env->tn;
  A.rho = rho;
  A.nn = env->h.nn;
  A.stats = env->stats;
  {
    LaunchTimer lt(env, st, FEMPIC_K_CHARGE);
    k_nodal_charge<<<blocks_for(p->n), kThreads, 0, st>>>(A);
    lt.kernels = 1;
  }
  FEMPIC_CUDA(cudaGetLastError());
  return FEMPIC_OK;
}

extern "C" int fempic_stats(fempic_env* env, int64_t* out4, void* stream) {
  if (!env || !out4) return fail(FEMPIC_EINVAL, "stats: NULL argument");
  unsigned long long h[3] = {0, 0, 0};
  cudaStream_t st = (cudaStream_t)stream;
  FEMPIC_CUDA(cudaMemcpyAsync(h, env->stats, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  FEMPIC_CUDA(cudaStreamSynchronize(st));
  out4[0] = (int64_t)h[0];
  out4[1] = (int64_t)h[1];
  out4[2] = env->steps;
  out4[3] = (int64_t)h[2];
  return FEMPIC_OK;
}

extern "C" int fempic_error_count(fempic_env* env, int64_t* n_bad, void* stream) {
  if (!env || !n_bad) return fail(FEMPIC_EINVAL, "error_count: NULL argument");
  unsigned long long h[4] = {0, 0, 0, 0};
  cudaStream_t st = (cudaStream_t)stream;
  FEMPIC_CUDA(cudaMemcpyAsync(h, env->stats, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  FEMPIC_CUDA(cudaStreamSynchronize(st));
  *n_bad = (int64_t)(h[1] - env->seen_frozen);
  const unsigned long long gave_up = h[2] - env->seen_timeouts;
  const unsigned long long bad_idx = h[3] - env->seen_bounds;
  env->seen_frozen = h[1];
  env->seen_timeouts = h[2];
  env->seen_bounds = h[3];
  if (gave_up)
    return fail(FEMPIC_EINCOMPLETE, "error_count: " + std::to_string(gave_up) +
                                        " staged push CTA(s) gave up waiting for a bulk copy; the particles of "
                                        "their remaining tiles were not advanced and their deposit is missing");
  if (bad_idx)
    return fail(FEMPIC_EBOUNDS, "error_count: " + std::to_string(bad_idx) +
                                    " mesh-table index(es) out of range were skipped (debug build)");
  return FEMPIC_OK;
}

extern "C" int fempic_debug_set_table(fempic_env* env, int32_t table, int64_t index, int32_t value) {
  if (!env) return fail(FEMPIC_EINVAL, "debug_set_table: NULL env");
  if (!kBoundsCheck)
    return fail(FEMPIC_EINVAL, "debug_set_table: only the debug build (FEMPIC_BOUNDS_CHECK) accepts it");
  const int64_t nt = env->h.nt;
  if (table == FEMPIC_TABLE_NEIGHBOUR) {
    if (index < 0 || index >= 4 * nt) return fail(FEMPIC_EINVAL, "debug_set_table: neighbour index out of range");
    // the neighbour table and its copy in the last 16 B of the tet record
    int32_t* nb = reinterpret_cast<int32_t*>(env->nb);
    FEMPIC_CUDA(cudaMemcpy(nb + index, &value, sizeof(int32_t), cudaMemcpyHostToDevice));
    float* rec = reinterpret_cast<float*>(env->tetrec);
    FEMPIC_CUDA(cudaMemcpy(rec + 32 * (index / 4) + 28 + index % 4, &value, sizeof(int32_t),
                           cudaMemcpyHostToDevice));
  } else if (table == FEMPIC_TABLE_EDGE) {
    if (index < 0 || index >= 6 * nt) return fail(FEMPIC_EINVAL, "debug_set_table: edge index out of range");
    int32_t* te = reinterpret_cast<int32_t*>(env->te);
    FEMPIC_CUDA(cudaMemcpy(te + 8 * (index / 6) + index % 6, &value, sizeof(int32_t), cudaMemcpyHostToDevice));
  } else {
    return fail(FEMPIC_EINVAL, "debug_set_table: unknown table");
  }
  return FEMPIC_OK;
}

extern "C" int fempic_debug_stall(fempic_env* env, int32_t cta, int64_t limit_ns) {
  if (!env) return fail(FEMPIC_EINVAL, "debug_stall: NULL env");
  if (cta < 0 || limit_ns < 1000 || limit_ns > (int64_t)kWaitLimitNs)
    return fail(FEMPIC_EINVAL, "debug_stall: cta >= 0 and 1 us <= limit_ns <= 1 s");
  env->stall_cta = cta;
  env->stall_ns = (unsigned long long)limit_ns;
  return FEMPIC_OK;
}

// ------------------------------------------------ measurement support
// FP64 FMA issue-rate probe: every thread runs `iters` rounds of 8
// independent FMA chains (no dependence between the chains, so the rate is
// the FP64 pipe's, not its latency); the result is stored only under a
// condition that never holds, which keeps the work from being removed.
__global__ void __launch_bounds__(kThreads) k_fp64_probe(int iters, double* out) {
  double a[8];
#pragma unroll
  for (int j = 0; j < 8; j++) a[j] = 1.0 + 1e-3 * (threadIdx.x + j);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < 8; j++) a[j] = fma(a[j], 0.9999999, 1e-7);
  }
  double sum = 0.0;
#pragma unroll
  for (int j = 0; j < 8; j++) sum += a[j];
  if (sum == -1.0) out[0] = sum;
}

extern "C" int fempic_measure_fp64_rate(double* lane_ops_per_s, void* stream) {
  if (!lane_ops_per_s) return fail(FEMPIC_EINVAL, "measure_fp64_rate: NULL output");
  int dev = 0, sms = 1;
  FEMPIC_CUDA(cudaGetDevice(&dev));
  FEMPIC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t st = (cudaStream_t)stream;
  double* sink = nullptr;
  FEMPIC_CUDA(cudaMalloc(&sink, sizeof(double)));
  cudaEvent_t a = nullptr, b = nullptr;
  int rc = FEMPIC_OK;
  const unsigned grid = (unsigned)sms * 8u;
  const int iters = 2048;
  float ms = 0.f;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    rc = fail(FEMPIC_ECUDA, "measure_fp64_rate: event creation");
  } else {
    k_fp64_probe<<<grid, kThreads, 0, st>>>(iters, sink);   // warm-up
    cudaEventRecord(a, st);
    k_fp64_probe<<<grid, kThreads, 0, st>>>(iters, sink);
    cudaEventRecord(b, st);
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess || !(ms > 0.f))
      rc = fail(FEMPIC_ECUDA, "measure_fp64_rate: timing");
    else
      *lane_ops_per_s = (double)grid * kThreads * iters * 8.0 / (ms * 1e-3);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(sink);
  return rc;
}

extern "C" int fempic_profile_enable(fempic_env* env, int32_t enable) {
  if (!env) return fail(FEMPIC_EINVAL, "profile_enable: NULL env");
  if (enable) {
    env->recs.clear();
    env->pool_used = 0;
  }
  env->profiling = enable != 0;
  return FEMPIC_OK;
}

extern "C" int fempic_profile_read(fempic_env* env, double* ms_out, int64_t* calls_out, int64_t* kernels_out) {
  if (!env || !ms_out || !calls_out || !kernels_out) return fail(FEMPIC_EINVAL, "profile_read: NULL argument");
  for (int k = 0; k < FEMPIC_K_COUNT; k++) {
    ms_out[k] = 0.0;
    calls_out[k] = 0;
    kernels_out[k] = 0;
  }
  for (const auto& r : env->recs) {
    FEMPIC_CUDA(cudaEventSynchronize(r.b));
    float ms = 0.f;
    FEMPIC_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    if (r.kid >= 0 && r.kid < FEMPIC_K_COUNT) {
      ms_out[r.kid] += ms;
      calls_out[r.kid]++;
      kernels_out[r.kid] += r.kernels;
    }
  }
  return FEMPIC_OK;
}

// Checks shared by the sort entry points: the two particle sets agree in
// size, species table and n_cross, do not overlap, and the key and particle
// counts fit 32-bit counters.  Sets *keys = n_species * (n_tets + 1).
static int sort_check(const char* name, fempic_env* env, const fempic_particles* in, const fempic_particles* out,
                      int64_t* keys) {
  const std::string nm(name);
  if (!env || !in || !out) return fail(FEMPIC_EINVAL, nm + ": NULL argument");
  int rc = check_particles(in, true);
  if (rc) return rc;
  rc = check_particles(out, true);
  if (rc) return rc;
  if (in->n != out->n || in->n_species != out->n_species || (!in->n_cross) != (!out->n_cross))
    return fail(FEMPIC_EINVAL, nm + ": in/out particle sets differ in size, species or n_cross");
  for (int s = 0; s <= in->n_species; s++)
    if (in->species_begin[s] != out->species_begin[s]) return fail(FEMPIC_EINVAL, nm + ": species tables differ");
  if (in->n > 0 && (in->x == out->x || in->tet == out->tet)) return fail(FEMPIC_EINVAL, nm + ": in and out overlap");
  *keys = (int64_t)in->n_species * (env->h.nt + 1);
  if (*keys >= (int64_t(1) << 31)) return fail(FEMPIC_EINVAL, nm + ": too many (species, tet) keys");
  if (in->n >= (int64_t(1) << 31)) return fail(FEMPIC_EINVAL, nm + ": more than 2^31 particles");
  return FEMPIC_OK;
}

// The counting sort by (species, tet) on caller-given scratch: counts and
// offsets [keys], sums [keys / (2 kScan) + 1].  Stream-ordered.
static int sort_launch(fempic_env* env, const fempic_particles* in, const fempic_particles* out, int32_t* perm,
                       int64_t k, int32_t* counts, int32_t* offsets, int32_t* sums, cudaStream_t st) {
  SortArgs A{};
  int rc = fill_species(in, 1.0, &A.sp);
  if (rc) return rc;
  const int64_t nt = env->h.nt;
  const int64_t tiles = (k + 2 * kScan - 1) / (2 * kScan);
  FEMPIC_CUDA(cudaMemsetAsync(counts, 0, k * sizeof(int32_t), st));
  k_sort_hist<<<blocks_for(in->n), kThreads, 0, st>>>(in->n, in->tet, A.sp, nt, counts);
  k_scan_tiles<<<(unsigned)tiles, kScan, 0, st>>>(k, counts, offsets, sums);
  k_scan_sums<<<1, kScan, 0, st>>>(tiles, sums);
  k_scan_add<<<blocks_for(k), kThreads, 0, st>>>(k, offsets, sums);
  FEMPIC_CUDA(cudaMemsetAsync(counts, 0, k * sizeof(int32_t), st));
  A.n = in->n;
  A.nt = nt;
  A.vbytes = env->opt.precision == FEMPIC_FP64 ? 8 : 4;
  A.x = in->x;
  A.y = in->y;
  A.z = in->z;
  A.vx = in->vx;
  A.vy = in->vy;
  A.vz = in->vz;
  A.tet = in->tet;
  A.status = in->status;
  A.ncross = in->n_cross;
  A.ox = out->x;
  A.oy = out->y;
  A.oz = out->z;
  A.ovx = out->vx;
  A.ovy = out->vy;
  A.ovz = out->vz;
  A.otet = out->tet;
  A.ostatus = out->status;
  A.oncross = out->n_cross;
  A.offsets = offsets;
  A.cursor = counts;
  A.operm = perm;
  k_sort_scatter<<<blocks_for(in->n), kThreads, 0, st>>>(A);
  FEMPIC_CUDA(cudaGetLastError());
  return FEMPIC_OK;
}

static int sort_impl(fempic_env* env, const fempic_particles* in, const fempic_particles* out, int32_t* perm,
                     void* stream) {
  int64_t k = 0;
  int rc = sort_check("sort", env, in, out, &k);
  if (rc || in->n == 0) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (env->sort_cap < k) {
    if (env->sort_counts) {
      FEMPIC_CUDA(cudaStreamSynchronize(st));
      cudaFree(env->sort_counts);
      cudaFree(env->sort_offsets);
      cudaFree(env->sort_sums);
      env->sort_counts = env->sort_offsets = env->sort_sums = nullptr;
      env->sort_cap = 0;
    }
    FEMPIC_CUDA(dalloc(&env->sort_counts, k));
    FEMPIC_CUDA(dalloc(&env->sort_offsets, k));
    FEMPIC_CUDA(dalloc(&env->sort_sums, k / (2 * kScan) + 1));
    env->sort_cap = k;
  }
  LaunchTimer lt(env, st, FEMPIC_K_SORT);
  lt.kernels = 5;   // histogram, three scan passes, scatter
  return sort_launch(env, in, out, perm, k, env->sort_counts, env->sort_offsets, env->sort_sums, st);
}

extern "C" int fempic_sort(fempic_env* env, const fempic_particles* in, const fempic_particles* out, void* stream) {
  return sort_impl(env, in, out, nullptr, stream);
}

extern "C" int fempic_sort_perm(fempic_env* env, const fempic_particles* in, const fempic_particles* out,
                                int32_t* perm, void* stream) {
  if (!perm) return fail(FEMPIC_EINVAL, "sort_perm: NULL permutation");
  return sort_impl(env, in, out, perm, stream);
}

extern "C" int fempic_adjoint_unpermute(fempic_env* env, const fempic_adjoint* in, const fempic_adjoint* out,
                                        const int32_t* perm, void* stream) {
  if (!env || !in || !out || !perm) return fail(FEMPIC_EINVAL, "adjoint_unpermute: NULL argument");
  if (in->n != out->n || in->n < 0) return fail(FEMPIC_EINVAL, "adjoint_unpermute: sizes differ");
  if (in->n == 0) return FEMPIC_OK;
  if (!in->rx || !in->ry || !in->rz || !in->vx || !in->vy || !in->vz || !out->rx || !out->ry || !out->rz ||
      !out->vx || !out->vy || !out->vz)
    return fail(FEMPIC_EINVAL, "adjoint_unpermute: NULL array");
  if (in->rx == out->rx || in->vx == out->vx) return fail(FEMPIC_EINVAL, "adjoint_unpermute: in and out overlap");
  if (in->n >= (int64_t(1) << 31)) return fail(FEMPIC_EINVAL, "adjoint_unpermute: more than 2^31 particles");
  AdjPermArgs A{};
  A.n = in->n;
  A.vbytes = env->opt.precision == FEMPIC_FP64 ? 8 : 4;
  A.perm = perm;
  A.rx = in->rx;
  A.ry = in->ry;
  A.rz = in->rz;
  A.vx = in->vx;
  A.vy = in->vy;
  A.vz = in->vz;
  A.ox = out->rx;
  A.oy = out->ry;
  A.oz = out->rz;
  A.ovx = out->vx;
  A.ovy = out->vy;
  A.ovz = out->vz;
  k_adjoint_unpermute<<<blocks_for(A.n), kThreads, 0, (cudaStream_t)stream>>>(A);
  FEMPIC_CUDA(cudaGetLastError());
  return FEMPIC_OK;
}

// ------------------------------------------------- sort without allocation
// Fixed scratch for fempic_sort_noalloc: per-key counters, per-key offsets
// and per-tile sums, sized for FEMPIC_SORT_NOALLOC_MAX_KEYS keys.
namespace {
constexpr int64_t kNoAllocKeys = FEMPIC_SORT_NOALLOC_MAX_KEYS;
constexpr int64_t kNoAllocTiles = kNoAllocKeys / (2 * kScan) + 1;
constexpr int kNoAllocMaxDevices = 64;
}  // namespace

static __device__ __align__(256) int32_t g_sort_noalloc_scratch[2 * kNoAllocKeys + kNoAllocTiles];

namespace {
std::mutex g_noalloc_mu;
int32_t* g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  In host code
// the symbol names a host-side shadow, so the address must come from
// cudaGetSymbolAddress, once per device, with that device current.
int noalloc_scratch(int32_t** out) {
  int dev = 0;
  FEMPIC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(FEMPIC_EINVAL, "sort_noalloc: device index too large");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    FEMPIC_CUDA(cudaGetSymbolAddress(&p, g_sort_noalloc_scratch));
    g_noalloc_addr[dev] = static_cast<int32_t*>(p);
  }
  *out = g_noalloc_addr[dev];
  return FEMPIC_OK;
}
}  // namespace

extern "C" int fempic_sort_noalloc(fempic_env* env, const fempic_particles* in, const fempic_particles* out,
                                   void* stream) {
  int64_t k = 0;
  int rc = sort_check("sort_noalloc", env, in, out, &k);
  if (rc || in->n == 0) return rc;
  if (k > kNoAllocKeys)
    return fail(FEMPIC_EINVAL, "sort_noalloc: n_species * (n_tets + 1) = " + std::to_string(k) +
                                   " exceeds the fixed scratch of " + std::to_string(kNoAllocKeys) +
                                   " keys; use fempic_sort");
  int32_t* base = nullptr;
  rc = noalloc_scratch(&base);
  if (rc) return rc;
  return sort_launch(env, in, out, nullptr, k, base, base + kNoAllocKeys, base + 2 * kNoAllocKeys,
                     (cudaStream_t)stream);
}

// ------------------------------------------------------------------ adjoint ABI
static int check_adjoint(const fempic_adjoint* a, int64_t n) {
  if (!a) return fail(FEMPIC_EINVAL, "adjoint: NULL adjoint state");
  if (a->n != n) return fail(FEMPIC_EINVAL, "adjoint: size differs from the particle set");
  if (n > 0 && (!a->rx || !a->ry || !a->rz || !a->vx || !a->vy || !a->vz))
    return fail(FEMPIC_EINVAL, "adjoint: NULL array");
  return FEMPIC_OK;
}

extern "C" int fempic_push_step_adjoint(fempic_env* env, const fempic_particles* before,
                                        const fempic_particles* after, const fempic_envelope* envl, double omega0,
                                        double t, double dt, const fempic_adjoint* adj, void* e_grad, void* b_grad,
                                        void* stream) {
  if (!env || !envl || !e_grad || !b_grad) return fail(FEMPIC_EINVAL, "push_step_adjoint: NULL argument");
  int rc = check_particles(before, true);
  if (rc) return rc;
  rc = check_particles(after, true);
  if (rc) return rc;
  if (before->n != after->n) return fail(FEMPIC_EINVAL, "push_step_adjoint: before/after sizes differ");
  rc = check_adjoint(adj, before->n);
  if (rc) return rc;
  if (!envl->e_tilde || !envl->b_tilde) return fail(FEMPIC_EINVAL, "push_step_adjoint: NULL DoF arrays");
  if (!(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(omega0) || !std::isfinite(t) || !std::isfinite(envl->amp))
    return fail(FEMPIC_EINVAL, "push_step_adjoint: non-finite or non-positive scalar");
  cudaStream_t st = (cudaStream_t)stream;
  AdjArgs A{};
  rc = fill_species(before, dt, &A.sp);
  if (rc) return rc;
  const bool mixed = env->opt.precision != FEMPIC_FP64;
  const int64_t nt = env->h.nt;
  if (!env->tetgrad) {
    FEMPIC_CUDA(dalloc(&env->tetgrad, 10 * nt));
    FEMPIC_CUDA(cudaMemsetAsync(env->tetgrad, 0, 10 * nt * sizeof(double), st));
  }
  if (mixed && !env->tetgrad32) {
    FEMPIC_CUDA(dalloc(&env->tetgrad32, 12 * nt));
    FEMPIC_CUDA(cudaMemsetAsync(env->tetgrad32, 0, 12 * nt * sizeof(float), st));
  }
  LaunchTimer lt(env, st, FEMPIC_K_ADJOINT);
  lt.kernels = 2;   // field, field adjoint (+ the particle adjoint below)
  // the per-tet affine field of this step (same carrier as the forward step)
  const double phi = omega0 * t;
  double cre = envl->amp * std::cos(phi), cim = envl->amp * std::sin(phi);
  if (mixed) {
    Levels<float2, float> L{};
    L.ne = env->h.ne;
    L.nf = env->h.nf;
    L.stats = env->stats;
    L.e[0] = static_cast<const float2*>(envl->e_tilde);
    L.b[0] = static_cast<const float2*>(envl->b_tilde);
    L.cre[0] = (float)cre;
    L.cim[0] = (float)cim;
    k_field_f32<1><<<blocks_for(nt), kThreads, 0, st>>>(nt, env->tetrec, env->te, env->tf, L);
    cre = (double)(float)cre;
    cim = (double)(float)cim;
  } else {
    Levels<double2, double> L{};
    L.ne = env->h.ne;
    L.nf = env->h.nf;
    L.stats = env->stats;
    L.e[0] = static_cast<const double2*>(envl->e_tilde);
    L.b[0] = static_cast<const double2*>(envl->b_tilde);
    L.cre[0] = cre;
    L.cim[0] = cim;
    k_field_fp64<1><<<blocks_for(nt), kThreads, 0, st>>>(nt, env->geom64, env->te, env->tf, L,
                                                          static_cast<double*>(env->field));
  }
  FEMPIC_CUDA(cudaGetLastError());
  if (before->n > 0) {
    A.n = before->n;
    A.x = before->x;
    A.y = before->y;
    A.z = before->z;
    A.vx = before->vx;
    A.vy = before->vy;
    A.vz = before->vz;
    A.tet = before->tet;
    A.vx1 = after->vx;
    A.vy1 = after->vy;
    A.vz1 = after->vz;
    A.status1 = after->status;
    A.dt = dt;
    A.nt = nt;
    A.geom64 = env->geom64;
    A.field64 = static_cast<const double*>(env->field);
    A.tetrec = env->tetrec;
    A.rbx = adj->rx;
    A.rby = adj->ry;
    A.rbz = adj->rz;
    A.vbx = adj->vx;
    A.vby = adj->vy;
    A.vbz = adj->vz;
    A.tetgrad = env->tetgrad;
    A.tetgrad32 = env->tetgrad32;
    A.curw = env->curw_on ? env->curw : nullptr;
    A.nb = env->nb;
    A.tn = env->tn;
    A.stats = env->stats;
    A.max_cross = env->opt.max_crossings;
    A.wall_mode = env->opt.wall_mode;
    for (int a = 0; a < 3; a++) {
      A.lo[a] = env->h.lo[a];
      A.hi[a] = env->h.hi[a];
    }
    if (mixed) {
      if (A.curw)
        k_push_adjoint<float, true><<<blocks_for(A.n), kThreads, 0, st>>>(A);
      else
        k_push_adjoint<float, false><<<blocks_for(A.n), kThreads, 0, st>>>(A);
    } else {
      if (A.curw)
        k_push_adjoint<double, true><<<blocks_for(A.n), kThreads, 0, st>>>(A);
      else
        k_push_adjoint<double, false><<<blocks_for(A.n), kThreads, 0, st>>>(A);
    }
    lt.kernels++;
    FEMPIC_CUDA(cudaGetLastError());
  }
  if (!env->tadj) FEMPIC_CUDA(dalloc(&env->tadj, 10 * nt));
  if (mixed)
    k_field_adjoint<float><<<blocks_for(nt), kThreads, 0, st>>>(nt, env->geom64, env->tetrec, env->tetgrad,
                                                                env->tetgrad32, env->tadj);
  else
    k_field_adjoint<double><<<blocks_for(nt), kThreads, 0, st>>>(nt, env->geom64, env->tetrec, env->tetgrad,
                                                                 env->tetgrad32, env->tadj);
  const int64_t ndof = std::max(env->h.ne, env->h.nf);
  k_dof_grad<<<blocks_for(ndof), kThreads, 0, st>>>(env->h.ne, env->h.nf, env->estart, env->eslot, env->fslot,
                                                     env->tadj, cre, cim, static_cast<double*>(e_grad),
                                                     static_cast<double*>(b_grad), nt, env->stats);
  lt.kernels++;
  FEMPIC_CUDA(cudaGetLastError());
  return FEMPIC_OK;
}

extern "C" int fempic_adjoint_current_weights(fempic_env* env, const double* u, void* stream) {
  if (!env) return fail(FEMPIC_EINVAL, "adjoint_current_weights: NULL env");
  if (!u) {
    env->curw_on = false;
    return FEMPIC_OK;
  }
  const int64_t nt = env->h.nt;
  if (!env->curw) FEMPIC_CUDA(dalloc(&env->curw, 6 * nt));
  cudaStream_t st = (cudaStream_t)stream;
  k_current_weights<<<blocks_for(nt), kThreads, 0, st>>>(nt, env->geom64, env->te, u, env->curw, env->h.ne,
                                                          env->stats);
  FEMPIC_CUDA(cudaGetLastError());
  env->curw_on = true;
  return FEMPIC_OK;
}

extern "C" int fempic_kinetic_energy(fempic_env* env, const fempic_particles* p, double* ke,
                                     const fempic_adjoint* seed, void* stream) {
  if (!env || !ke) return fail(FEMPIC_EINVAL, "kinetic_energy: NULL argument");
  int rc = check_particles(p, true);
  if (rc) return rc;
  if (seed) {
    rc = check_adjoint(seed, p->n);
    if (rc) return rc;
  }
  cudaStream_t st = (cudaStream_t)stream;
  FEMPIC_CUDA(cudaMemsetAsync(ke, 0, sizeof(double), st));
  if (p->n == 0) return FEMPIC_OK;
  KEArgs A{};
  rc = fill_species(p, 1.0, &A.sp);
  if (rc) return rc;
  for (int s = 0; s < kMaxSpecies; s++) A.mw[s] = s < p->n_species ? p->m[s] * p->w[s] : 0.0;
  A.n = p->n;
  A.vx = p->vx;
  A.vy = p->vy;
  A.vz = p->vz;
  A.tet = p->tet;
  A.ke = ke;
  if (seed) {
    A.rbx = seed->rx;
    A.rby = seed->ry;
    A.rbz = seed->rz;
    A.vbx = seed->vx;
    A.vby = seed->vy;
    A.vbz = seed->vz;
  }
  if (env->opt.precision != FEMPIC_FP64)
    k_kinetic_energy<float><<<blocks_for(p->n), kThreads, 0, st>>>(A);
  else
    k_kinetic_energy<double><<<blocks_for(p->n), kThreads, 0, st>>>(A);
  FEMPIC_CUDA(cudaGetLastError());
  return FEMPIC_OK;
}
