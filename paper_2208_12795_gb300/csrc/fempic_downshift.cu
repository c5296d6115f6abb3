// Downshifted particle integrator of Sec. III-D on the FP64 form and the
// FP32-mixed forms: the velocity rule with the carrier integrated
// analytically (M and L weights) and AB4 positions.  Per step: k_ds_field (per-tet envelope coefficients),
// k_ds_pre (sample, velocity rule, AB4 velocity, history shift), the env's
// own FP64 step under a zero field (tracking, walls, deposit of the AB4
// segment), then k_ds_post (wall mirrors of the velocity history).
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <string>

#include "fempic_downshift.h"
#include "fempic_internal.h"

namespace {

using fempic::HostMesh;
using fempic::kMaxSpecies;

thread_local std::string g_ds_error;

int fail(int code, const std::string& msg) {
  g_ds_error = msg;
  return code;
}

#define DS_CUDA(call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return fail(FEMPIC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

constexpr int kThreads = 256;

// Fourth-order Adams-Bashforth stencil (55, -59, 37, -9) / 24, divided once
// here: a double division per particle costs several FP64-pipe instructions.
__device__ constexpr double kAB4[4] = {55.0 / 24.0, -59.0 / 24.0, 37.0 / 24.0, -9.0 / 24.0};

// Local edge e joins sorted local nodes (le0, le1) in the order 01,02,03,12,
// 13,23; local face f is opposite node f and its i-th node is lf(f, i).
__host__ __device__ constexpr int le0(int e) { return e < 3 ? 0 : (e < 5 ? 1 : 2); }
__host__ __device__ constexpr int le1(int e) { return e < 3 ? e + 1 : (e == 3 ? 2 : 3); }
__host__ __device__ constexpr int lf(int f, int i) { return i < f ? i : i + 1; }

// Debug build (FEMPIC_BOUNDS_CHECK): an edge or face id read from this unit's
// tables is checked against its range before it addresses a DoF array; an
// out-of-range id is counted in the env's bounds counter (reported by
// fempic_error_count) and its DoF reads as zero.
#ifdef FEMPIC_BOUNDS_CHECK
constexpr bool kBoundsCheck = true;
#else
constexpr bool kBoundsCheck = false;
#endif
__device__ __forceinline__ bool ds_idx_in(int64_t i, int64_t n, unsigned long long* stats) {
  if (!kBoundsCheck) return true;
  if (i >= 0 && i < n) return true;
  if (stats) atomicAdd(stats + 3, 1ull);
  return false;
}

struct DsArgs {
  int64_t n;
  const double* x;
  const double* y;
  const double* z;
  void* vx;                     // f64 (FP64 form) or f32 (mixed forms) velocities
  void* vy;
  void* vz;
  const int32_t* tet;
  void* h;                      // history planes [FEMPIC_DS_PLANES][n], the velocity type
  int64_t nt;
  const double* geom;           // [nt][12]: x0, grad l1, grad l2, grad l3
  const double* coef;           // [nt][20]: per-tet envelope coefficients of this step (k_ds_field)
  const float* coef32;          // mixed forms: the same in FP32
  int32_t ns;
  int32_t start;
  int64_t begin[kMaxSpecies + 1];
  double qm[kMaxSpecies];
  double w[24];                 // M^r[3], M^i[3], L^r[3][3], L^i[3][3]
  float qm32[kMaxSpecies];      // mixed forms: the same rounded to FP32
  float w32[24];
};

__device__ __forceinline__ int species_of(const DsArgs& A, int64_t p) {
  int s = 0;
#pragma unroll 1
  while (s + 1 < A.ns && p >= A.begin[s + 1]) s++;
  return s;
}

template <typename R>
__device__ __forceinline__ void cross3(const R a[3], const R b[3], R o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// Per-tet complex envelope coefficients of one step (Sec. III-A).  Inside a
// tet both Whitney sums are affine in d = r - x0 (x0 = the tet's node 0,
// lambda_k = delta_k0 + g_k . d with g_k = grad lambda_k):
//   W1_ij = const + d x (g_j x g_i), so E~ = E0 + d x W with
//     E0 = sum_j e~_0j g_j,  W = sum_{i<j} e~_ij (g_j x g_i);
//   W2_ijk = const + 2 det[g_i, g_j, g_k] d, so B~ = B0 + beta d with
//     B0 = 2 sum over the faces (0, j, k) of b~_f g_j x g_k,
//     beta = 2 sum_f b~_f det[g_i, g_j, g_k].
// coef[20 t ..]: Re (E0, W, B0, beta), then Im (E0, W, B0, beta), times a(t).
template <typename C2>
__global__ void __launch_bounds__(kThreads) k_ds_field(int64_t nt, const double* __restrict__ geom,
                                                       const int32_t* __restrict__ te,
                                                       const int32_t* __restrict__ tf,
                                                       const C2* __restrict__ e,
                                                       const C2* __restrict__ b, int64_t ne, int64_t nf,
                                                       unsigned long long* stats, double amp,
                                                       double* __restrict__ coef, float* __restrict__ coef32) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const double* G = geom + 12 * t;
  double g[4][3];
#pragma unroll
  for (int k = 1; k < 4; k++)
#pragma unroll
    for (int a = 0; a < 3; a++) g[k][a] = G[3 * k + a];
#pragma unroll
  for (int a = 0; a < 3; a++) g[0][a] = -(g[1][a] + g[2][a] + g[3][a]);
  double o[20];
#pragma unroll
  for (int c = 0; c < 20; c++) o[c] = 0.0;
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const int i = le0(k), j = le1(k);
    const int32_t id = te[6 * t + k];
    double2 c = make_double2(0.0, 0.0);
    if (ds_idx_in(id, ne, stats)) {
      const C2 cc = e[id];
      c = make_double2((double)cc.x, (double)cc.y);
    }
    double gji[3];
    cross3(g[j], g[i], gji);
#pragma unroll
    for (int a = 0; a < 3; a++) {
      if (i == 0) {
        o[a] += c.x * g[j][a];
        o[10 + a] += c.y * g[j][a];
      }
      o[3 + a] += c.x * gji[a];
      o[13 + a] += c.y * gji[a];
    }
  }
#pragma unroll
  for (int f = 0; f < 4; f++) {
    const int i = lf(f, 0), j = lf(f, 1), k = lf(f, 2);
    const int32_t id = tf[4 * t + f];
    double2 c = make_double2(0.0, 0.0);
    if (ds_idx_in(id, nf, stats)) {
      const C2 cc = b[id];
      c = make_double2((double)cc.x, (double)cc.y);
    }
    double gjk[3];
    cross3(g[j], g[k], gjk);
    const double det = g[i][0] * gjk[0] + g[i][1] * gjk[1] + g[i][2] * gjk[2];
    if (i == 0) {
#pragma unroll
      for (int a = 0; a < 3; a++) {
        o[6 + a] += 2.0 * c.x * gjk[a];
        o[16 + a] += 2.0 * c.y * gjk[a];
      }
    }
    o[9] += 2.0 * c.x * det;
    o[19] += 2.0 * c.y * det;
  }
  double2* out = reinterpret_cast<double2*>(coef + 20 * t);
#pragma unroll
  for (int c = 0; c < 10; c++) out[c] = make_double2(amp * o[2 * c], amp * o[2 * c + 1]);
  if (coef32) {
    float2* o32 = reinterpret_cast<float2*>(coef32 + 20 * t);
#pragma unroll
    for (int c = 0; c < 10; c++) o32[c] = make_float2((float)(amp * o[2 * c]), (float)(amp * o[2 * c + 1]));
  }
}

// The envelope sample at r in tet T from the per-tet coefficients:
// out[12] = Re E~, Im E~, Re B~, Im B~.  The mixed forms take d = r - x0 from
// one FP64 subtraction, rounded to FP32, and evaluate in FP32.
template <typename R>
__device__ __forceinline__ void envelope_at(const DsArgs& A, int32_t T, double rx, double ry, double rz,
                                            R out[12]) {
  const double* G = A.geom + 12 * (int64_t)T;
  const R d[3] = {(R)(rx - __ldg(G)), (R)(ry - __ldg(G + 1)), (R)(rz - __ldg(G + 2))};
  R c[20];
  if (sizeof(R) == 8) {
    const double2* C = reinterpret_cast<const double2*>(A.coef + 20 * (int64_t)T);
#pragma unroll
    for (int i = 0; i < 10; i++) {
      const double2 v = __ldg(C + i);
      c[2 * i] = (R)v.x;
      c[2 * i + 1] = (R)v.y;
    }
  } else {
    const float2* C = reinterpret_cast<const float2*>(A.coef32 + 20 * (int64_t)T);
#pragma unroll
    for (int i = 0; i < 10; i++) {
      const float2 v = __ldg(C + i);
      c[2 * i] = (R)v.x;
      c[2 * i + 1] = (R)v.y;
    }
  }
#pragma unroll
  for (int part = 0; part < 2; part++) {
    const R* q = c + 10 * part;
    R dw[3];
    cross3<R>(d, q + 3, dw);
#pragma unroll
    for (int a = 0; a < 3; a++) {
      out[3 * part + a] = q[a] + dw[a];
      out[6 + 3 * part + a] = q[6 + a] + q[9] * d[a];
    }
  }
}

// Before the env's step: the envelope sample at r^n, the velocity rule, the
// AB4 velocity u (left in v for the env's zero-field step to track), the new
// velocity and u kept in the scratch planes, and the history shifted.
// The FP32 instance streams the history planes and is bound by HBM latency:
// it is held to 80 registers so that 3 blocks of 256 stay resident per SM
// (128 registers left 2, and the step 4% slower).  The FP64 instance is bound
// by the FP64 pipe and keeps the compiler's allocation (a minimum of 0 leaves
// it unconstrained; 1 let it grow to 204 registers and one block per SM).
template <typename R>
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 3 : 0) k_ds_pre(DsArgs A) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= A.n) return;
  const int64_t n = A.n;
  R* H = static_cast<R*>(A.h);
  R* vxp = static_cast<R*>(A.vx);
  R* vyp = static_cast<R*>(A.vy);
  R* vzp = static_cast<R*>(A.vz);
  const R v0[3] = {vxp[p], vyp[p], vzp[p]};
  const int32_t T = A.tet[p];
  if (T < 0 || T >= A.nt) {   // inactive: the state is kept (the env's step flags an out-of-range tet)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      H[(FEMPIC_DS_VN + a) * n + p] = v0[a];
      H[(FEMPIC_DS_U + a) * n + p] = v0[a];
    }
    return;
  }
  R cur[12];
  envelope_at<R>(A, T, A.x[p], A.y[p], A.z[p], cur);
  R vh[3][3], f1[12], f2[12];
  if (A.start) {
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
      for (int a = 0; a < 3; a++) vh[i][a] = v0[a];
#pragma unroll
    for (int c = 0; c < 12; c++) f1[c] = f2[c] = cur[c];
  } else {
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
      for (int a = 0; a < 3; a++) vh[i][a] = H[(FEMPIC_DS_VH + 3 * i + a) * n + p];
#pragma unroll
    for (int c = 0; c < 12; c++) {
      f1[c] = H[(FEMPIC_DS_F + c) * n + p];
      f2[c] = H[(FEMPIC_DS_F + 12 + c) * n + p];
    }
  }
  const R* S[3] = {cur, f1, f2};
  const R* V[3] = {v0, vh[0], vh[1]};
  // weights from the kernel parameters: M^r at 0, M^i at 3, L^r at 6, L^i at 15
  auto wt = [&](int i) -> R { return sizeof(R) == 8 ? (R)A.w[i] : (R)A.w32[i]; };
  R dv[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int a = 0; a < 3; a++) dv[a] += S[k][a] * wt(k) + S[k][3 + a] * wt(3 + k);
#pragma unroll
  for (int j = 0; j < 3; j++) {
    R C[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
      for (int a = 0; a < 3; a++) C[a] += S[k][6 + a] * wt(6 + 3 * j + k) + S[k][9 + a] * wt(15 + 3 * j + k);
    R vc[3];
    cross3<R>(V[j], C, vc);
#pragma unroll
    for (int a = 0; a < 3; a++) dv[a] += vc[a];
  }
  const int s = species_of(A, p);
  const R qm = sizeof(R) == 8 ? (R)A.qm[s] : (R)A.qm32[s];
  const R ab[4] = {(R)kAB4[0], (R)kAB4[1], (R)kAB4[2], (R)kAB4[3]};
  R u[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    u[a] = ab[0] * v0[a] + ab[1] * vh[0][a] + ab[2] * vh[1][a] + ab[3] * vh[2][a];
    H[(FEMPIC_DS_VN + a) * n + p] = v0[a] + qm * dv[a];
    H[(FEMPIC_DS_U + a) * n + p] = u[a];
    H[(FEMPIC_DS_VH + 6 + a) * n + p] = vh[1][a];
    H[(FEMPIC_DS_VH + 3 + a) * n + p] = vh[0][a];
    H[(FEMPIC_DS_VH + a) * n + p] = v0[a];
  }
#pragma unroll
  for (int c = 0; c < 12; c++) {
    H[(FEMPIC_DS_F + 12 + c) * n + p] = f1[c];
    H[(FEMPIC_DS_F + c) * n + p] = cur[c];
  }
  vxp[p] = u[0];
  vyp[p] = u[1];
  vzp[p] = u[2];
}

// After the env's step: an axis in which the tracked velocity came back
// negated was mirrored by a wall (an odd number of times; a zero component
// cannot reach a wall), so the new velocity and the velocity history are
// mirrored in it; then v <- v^{n+1}.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_ds_post(DsArgs A) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= A.n) return;
  const int64_t n = A.n;
  R* H = static_cast<R*>(A.h);
  R* vp[3] = {static_cast<R*>(A.vx), static_cast<R*>(A.vy), static_cast<R*>(A.vz)};
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const R va = vp[a][p];
    const R u = H[(FEMPIC_DS_U + a) * n + p];
    R vn = H[(FEMPIC_DS_VN + a) * n + p];
    if (u != R(0) && va == -u) {
      vn = -vn;
#pragma unroll
      for (int i = 0; i < 3; i++) {
        R& h = H[(FEMPIC_DS_VH + 3 * i + a) * n + p];
        h = -h;
      }
    }
    vp[a][p] = vn;
  }
}

// int_0^1 x^m e^{j theta x} dx, m = 0..4: the power series of the exponential
// integrated term by term for |theta| <= 1, else the integration-by-parts
// recurrence J_m = (e^{j theta} - m J_{m-1}) / (j theta).
void moments(double theta, std::complex<double> J[5]) {
  using cd = std::complex<double>;
  if (std::fabs(theta) <= 1.0) {
    for (int m = 0; m < 5; m++) {
      cd term(1.0, 0.0), sum(0.0, 0.0);   // term = (j theta)^l / l!
      for (int l = 0; l < 40; l++) {
        sum += term / double(m + l + 1);
        term *= cd(0.0, theta) / double(l + 1);
      }
      J[m] = sum;
    }
  } else {
    const cd e = std::polar(1.0, theta), jt(0.0, theta);
    J[0] = (e - 1.0) / jt;
    for (int m = 1; m < 5; m++) J[m] = (e - double(m) * J[m - 1]) / jt;
  }
}

void compute_weights(double t, double dt, double omega0, double* w) {
  using cd = std::complex<double>;
  // basis on the nodes x_k = -k (x = (t' - t) / dt) as coefficient vectors
  double c[3][3];
  for (int k = 0; k < 3; k++) {
    double poly[3] = {1.0, 0.0, 0.0};
    for (int j = 0; j < 3; j++) {
      if (j == k) continue;
      const double xk = -double(k), xj = -double(j), den = xk - xj;
      double nxt[3] = {0.0, 0.0, 0.0};   // poly * (x - xj) / den
      for (int m = 0; m < 3; m++) {
        if (m + 1 < 3) nxt[m + 1] += poly[m] / den;
        nxt[m] -= poly[m] * xj / den;
      }
      for (int m = 0; m < 3; m++) poly[m] = nxt[m];
    }
    for (int m = 0; m < 3; m++) c[k][m] = poly[m];
  }
  cd J[5];
  moments(omega0 * dt, J);
  const cd f = dt * std::polar(1.0, omega0 * t);
  for (int k = 0; k < 3; k++) {
    cd I(0.0, 0.0);
    for (int m = 0; m < 3; m++) I += c[k][m] * J[m];
    I *= f;
    w[k] = I.real();
    w[3 + k] = -I.imag();
  }
  for (int j = 0; j < 3; j++)
    for (int k = 0; k < 3; k++) {
      double prod[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) prod[a + b] += c[j][a] * c[k][b];
      cd I(0.0, 0.0);
      for (int m = 0; m < 5; m++) I += prod[m] * J[m];
      I *= f;
      w[6 + 3 * j + k] = I.real();
      w[15 + 3 * j + k] = -I.imag();
    }
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

struct fempic_downshift {
  int64_t nn = 0, ne = 0, nf = 0, nt = 0;
  double* geom = nullptr;
  int32_t* te = nullptr;
  int32_t* tf = nullptr;
  double* coef = nullptr;       // [nt][20]
  float* coef32 = nullptr;      // mixed forms: [nt][20] in FP32 (allocated on first use)
};

static void free_ds(fempic_downshift* d) {
  if (!d) return;
  cudaFree(d->geom);
  cudaFree(d->te);
  cudaFree(d->tf);
  cudaFree(d->coef);
  cudaFree(d->coef32);
  delete d;
}

// History planes follow a particle sort: out[k][q] = in[k][perm[q]] for the
// planes that outlive a step (velocities and envelope samples; the two
// scratch vectors are rewritten by every step).
template <typename R>
__global__ void __launch_bounds__(kThreads) k_ds_permute(int64_t n, const int32_t* __restrict__ perm,
                                                          const R* __restrict__ in, R* __restrict__ out) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int64_t src = perm[q];
#pragma unroll 3
  for (int k = 0; k < FEMPIC_DS_VN; k++) out[k * n + q] = __ldg(in + k * n + src);
}

extern "C" const char* fempic_downshift_last_error(void) { return g_ds_error.c_str(); }

extern "C" int fempic_downshift_permute(const fempic_downshift_history* in, const fempic_downshift_history* out,
                                        const int32_t* perm, void* stream) {
  if (!in || !out || !perm) return fail(FEMPIC_EINVAL, "downshift_permute: NULL argument");
  if (in->n != out->n || in->n < 0) return fail(FEMPIC_EINVAL, "downshift_permute: sizes differ");
  if (in->n == 0) return FEMPIC_OK;
  if (!in->planes || !out->planes || in->planes == out->planes)
    return fail(FEMPIC_EINVAL, "downshift_permute: NULL or overlapping planes");
  if (in->f32 != out->f32 || (in->f32 != 0 && in->f32 != 1))
    return fail(FEMPIC_EINVAL, "downshift_permute: plane types differ");
  if (in->n >= (int64_t(1) << 31)) return fail(FEMPIC_EINVAL, "downshift_permute: more than 2^31 particles");
  const unsigned blocks = (unsigned)((in->n + kThreads - 1) / kThreads);
  if (in->f32)
    k_ds_permute<float><<<blocks, kThreads, 0, (cudaStream_t)stream>>>(
        in->n, perm, static_cast<const float*>(in->planes), static_cast<float*>(out->planes));
  else
    k_ds_permute<double><<<blocks, kThreads, 0, (cudaStream_t)stream>>>(
        in->n, perm, static_cast<const double*>(in->planes), static_cast<double*>(out->planes));
  DS_CUDA(cudaGetLastError());
  return FEMPIC_OK;
}

extern "C" void fempic_downshift_destroy(fempic_downshift* ds) { free_ds(ds); }

extern "C" int fempic_downshift_debug_set_table(fempic_downshift* ds, int32_t table, int64_t index,
                                                int32_t value) {
  if (!ds) return fail(FEMPIC_EINVAL, "downshift_debug_set_table: NULL handle");
  if (!kBoundsCheck)
    return fail(FEMPIC_EINVAL, "downshift_debug_set_table: only the debug build (FEMPIC_BOUNDS_CHECK) accepts it");
  int32_t* dst = nullptr;
  if (table == FEMPIC_TABLE_EDGE) {
    if (index < 0 || index >= 6 * ds->nt) return fail(FEMPIC_EINVAL, "downshift_debug_set_table: edge index out of range");
    dst = ds->te + index;
  } else if (table == FEMPIC_TABLE_FACE) {
    if (index < 0 || index >= 4 * ds->nt) return fail(FEMPIC_EINVAL, "downshift_debug_set_table: face index out of range");
    dst = ds->tf + index;
  } else {
    return fail(FEMPIC_EINVAL, "downshift_debug_set_table: unknown table");
  }
  DS_CUDA(cudaMemcpy(dst, &value, sizeof(int32_t), cudaMemcpyHostToDevice));
  return FEMPIC_OK;
}

extern "C" int fempic_downshift_create(const fempic_mesh_desc* mesh, fempic_downshift** out) {
  if (!mesh || !out) return fail(FEMPIC_EINVAL, "downshift_create: NULL argument");
  *out = nullptr;
  HostMesh m;
  std::string err;
  const int rc = fempic::build_host_mesh(*mesh, &m, &err);
  if (rc != FEMPIC_OK) return fail(rc, "downshift_create: " + err);
  fempic_downshift* d = new (std::nothrow) fempic_downshift();
  if (!d) return fail(FEMPIC_ENOMEM, "downshift_create: host allocation");
  d->nn = m.nn;
  d->ne = m.ne;
  d->nf = m.nf;
  d->nt = m.nt;
  const size_t sg = sizeof(double) * 12 * (size_t)m.nt, se = sizeof(int32_t) * 6 * (size_t)m.nt,
               sf = sizeof(int32_t) * 4 * (size_t)m.nt;
  if (cudaMalloc(&d->geom, sg) != cudaSuccess || cudaMalloc(&d->te, se) != cudaSuccess ||
      cudaMalloc(&d->tf, sf) != cudaSuccess ||
      cudaMalloc(&d->coef, sizeof(double) * 20 * (size_t)m.nt) != cudaSuccess) {
    free_ds(d);
    cudaGetLastError();
    return fail(FEMPIC_ENOMEM, "downshift_create: device allocation");
  }
  if (cudaMemcpy(d->geom, m.geom.data(), sg, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d->te, m.te.data(), se, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d->tf, m.tf.data(), sf, cudaMemcpyHostToDevice) != cudaSuccess) {
    free_ds(d);
    return fail(FEMPIC_ECUDA, "downshift_create: upload");
  }
  *out = d;
  return FEMPIC_OK;
}

extern "C" int fempic_downshift_weights(double t, double dt, double omega0, double* w_out) {
  if (!w_out) return fail(FEMPIC_EINVAL, "downshift_weights: NULL output");
  if (!std::isfinite(t) || !std::isfinite(dt) || !std::isfinite(omega0) || !(dt > 0.0))
    return fail(FEMPIC_EINVAL, "downshift_weights: non-finite scalar or dt <= 0");
  compute_weights(t, dt, omega0, w_out);
  return FEMPIC_OK;
}

extern "C" int fempic_push_step_downshift(fempic_env* env, fempic_downshift* ds, const fempic_particles* p,
                                          const fempic_downshift_history* hist, const fempic_envelope* envl,
                                          double omega0, double t, double dt, int32_t start, void* stream) {
  if (!env || !ds || !p || !hist || !envl) return fail(FEMPIC_EINVAL, "push_step_downshift: NULL argument");
  if (p->n < 0 || hist->n != p->n) return fail(FEMPIC_EINVAL, "push_step_downshift: history size != particles");
  if (!envl->e_tilde || !envl->b_tilde) return fail(FEMPIC_EINVAL, "push_step_downshift: NULL DoF arrays");
  if (!std::isfinite(t) || !std::isfinite(dt) || !(dt > 0.0) || !std::isfinite(omega0) ||
      !std::isfinite(envl->amp))
    return fail(FEMPIC_EINVAL, "push_step_downshift: non-finite scalar or dt <= 0");
  if (start != 0 && start != 1) return fail(FEMPIC_EINVAL, "push_step_downshift: start must be 0 or 1");
  const bool mixed = fempic::env_precision(env) != FEMPIC_FP64;
  if (hist->f32 != (mixed ? 1 : 0))
    return fail(FEMPIC_EINVAL, "push_step_downshift: history planes must be f64 for an FP64-form env and f32 "
                               "for a mixed-form env (fempic_downshift_history.f32)");
  // the env step it runs checks its arguments only after this step has
  // launched its own kernels: run those checks first, so that an error
  // leaves the particles and the history untouched
  if (fempic::validate_push_step(p, envl, omega0, t, dt) != FEMPIC_OK)
    return fail(FEMPIC_EINVAL, std::string("push_step_downshift: ") + fempic_last_error());
  int64_t counts[4];
  if (fempic_env_query(env, counts, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr) != FEMPIC_OK ||
      counts[3] != ds->nt || counts[1] != ds->ne || counts[2] != ds->nf)
    return fail(FEMPIC_EINVAL, "push_step_downshift: env and downshift tables are of different meshes");
  if (p->n == 0) return FEMPIC_OK;
  if (!hist->planes || !p->x || !p->y || !p->z || !p->vx || !p->vy || !p->vz || !p->tet || !p->status)
    return fail(FEMPIC_EINVAL, "push_step_downshift: NULL particle or history array");
  if (p->n_species < 1 || p->n_species > kMaxSpecies || !p->species_begin || !p->q || !p->m)
    return fail(FEMPIC_EINVAL, "push_step_downshift: species table (1..8 ranges, q, m)");
  if (p->species_begin[0] != 0 || p->species_begin[p->n_species] != p->n)
    return fail(FEMPIC_EINVAL, "push_step_downshift: species ranges must cover [0, n)");
  DsArgs A{};
  A.ns = p->n_species;
  for (int s = 0; s <= kMaxSpecies; s++) A.begin[s] = s <= p->n_species ? p->species_begin[s] : p->n;
  for (int s = 0; s < p->n_species; s++) {
    if (s > 0 && A.begin[s] < A.begin[s - 1]) return fail(FEMPIC_EINVAL, "push_step_downshift: species ranges decrease");
    if (!(p->m[s] > 0.0) || !std::isfinite(p->q[s])) return fail(FEMPIC_EINVAL, "push_step_downshift: q, m");
    A.qm[s] = p->q[s] / p->m[s];
    A.qm32[s] = (float)A.qm[s];
  }
  if (A.begin[p->n_species] < A.begin[p->n_species - 1])
    return fail(FEMPIC_EINVAL, "push_step_downshift: species ranges decrease");
  A.n = p->n;
  A.x = p->x;
  A.y = p->y;
  A.z = p->z;
  A.vx = p->vx;
  A.vy = p->vy;
  A.vz = p->vz;
  A.tet = p->tet;
  A.h = hist->planes;
  A.nt = ds->nt;
  A.geom = ds->geom;
  A.coef = ds->coef;
  A.start = start;
  compute_weights(t, dt, omega0, A.w);
  for (int i = 0; i < 24; i++) A.w32[i] = (float)A.w[i];
  if (mixed && !ds->coef32) {
    if (cudaMalloc(&ds->coef32, sizeof(float) * 20 * (size_t)ds->nt) != cudaSuccess) {
      cudaGetLastError();
      ds->coef32 = nullptr;
      return fail(FEMPIC_ENOMEM, "push_step_downshift: device allocation");
    }
  }
  A.coef32 = ds->coef32;
  cudaStream_t st = (cudaStream_t)stream;
  if (mixed) {   // complex64 DoFs; FP32 velocities, samples and history
    k_ds_field<float2><<<blocks_for(ds->nt), kThreads, 0, st>>>(
        ds->nt, ds->geom, ds->te, ds->tf, static_cast<const float2*>(envl->e_tilde),
        static_cast<const float2*>(envl->b_tilde), ds->ne, ds->nf, fempic::env_stats(env), envl->amp, ds->coef,
        ds->coef32);
    DS_CUDA(cudaGetLastError());
    k_ds_pre<float><<<blocks_for(p->n), kThreads, 0, st>>>(A);
  } else {
    k_ds_field<double2><<<blocks_for(ds->nt), kThreads, 0, st>>>(
        ds->nt, ds->geom, ds->te, ds->tf, static_cast<const double2*>(envl->e_tilde),
        static_cast<const double2*>(envl->b_tilde), ds->ne, ds->nf, fempic::env_stats(env), envl->amp, ds->coef,
        nullptr);
    DS_CUDA(cudaGetLastError());
    k_ds_pre<double><<<blocks_for(p->n), kThreads, 0, st>>>(A);
  }
  DS_CUDA(cudaGetLastError());
  // the AB4 segment: the env's own step under a zero field tracks, reflects
  // or absorbs and deposits r^n -> r^n + dt u
  fempic_envelope zero = *envl;
  zero.amp = 0.0;
  const int rc = fempic_push_step(env, p, &zero, omega0, t, dt, stream);
  if (rc != FEMPIC_OK) return fail(rc, std::string("push_step_downshift: env step: ") + fempic_last_error());
  if (mixed)
    k_ds_post<float><<<blocks_for(p->n), kThreads, 0, st>>>(A);
  else
    k_ds_post<double><<<blocks_for(p->n), kThreads, 0, st>>>(A);
  DS_CUDA(cudaGetLastError());
  return FEMPIC_OK;
}
