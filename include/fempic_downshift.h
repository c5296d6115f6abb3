/*
 * fempic_downshift.h -- C ABI of the downshifted particle integrator of
 * Sec. III-D (Ramachandran et al., "An Envelope Tracking Approach for
 * Particle in Cell Simulations"), on the FP64 form of fempic_env.h and on its
 * FP32-mixed forms (the rule, the samples and the history in FP32, positions
 * in FP64, the segment tracked and deposited by the env's mixed step).
 *
 * Over one particle step [t_n, t_n + dt] the Lorentz force is integrated with
 * the fast carrier treated analytically: the slowly varying envelope samples
 * of the last three steps are interpolated in time by the quadratic Lagrange
 * basis N_k, and the carrier enters only through the integrals
 *   M^r_k  =  int N_k cos(w0 t) dt,       M^i_k  = -int N_k sin(w0 t) dt,
 *   L^r_jk =  int N_j N_k cos(w0 t) dt,   L^i_jk = -int N_j N_k sin(w0 t) dt
 * (Sec. III-D, definitions of the M and L operators).  Per particle:
 *   v^{n+1} = v^n + (q/m) sum_k [Re(E~_k) M^r_k + Im(E~_k) M^i_k]
 *               + (q/m) sum_j sum_k v_j x [Re(B~_k) L^r_jk + Im(B~_k) L^i_jk]
 *   r^{n+1} = r^n + dt u,  u = (55 v^n - 59 v^{n-1} + 37 v^{n-2} - 9 v^{n-3}) / 24
 * (Sec. III-D, velocity rule and the fourth-order Adams-Bashforth position
 * stencil).  Sample k = 0, 1, 2 is level n - k: the complex envelope
 * E~ = sum_e e~_e W1_e, B~ = sum_f b~_f W2_f at the particle's position of
 * that level, times the slow amplitude a(t) of that level, and v_j = v^{n-j}.
 * The printed velocity rule is garbled in its level indices and uses the
 * two-index L with one index; the reading above (newest three samples, the
 * velocity and B~ interpolated separately) is the one implemented.
 *
 * The straight segment r^n -> r^{n+1} is tracked, reflected or absorbed at
 * the walls and deposited by the env's own FP64 step (fempic_push_step of
 * fempic_env.h run with a zero field, whose Boris update then leaves the
 * velocity unchanged).  A wall that mirrors the segment in an axis mirrors,
 * in that axis, the new velocity and every stored velocity of the history.
 *
 * Conventions: as in fempic_env.h (device / host pointers as stated, stream-
 * ordered asynchronous calls, FEMPIC_OK or a negative FEMPIC_E* code; the
 * message of the last failure of these entry points on the calling thread is
 * fempic_downshift_last_error()).
 */
#ifndef FEMPIC_DOWNSHIFT_H
#define FEMPIC_DOWNSHIFT_H

#include "fempic_env.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fempic_downshift fempic_downshift;   /* opaque: per-tet geometry, edge and face
                                                       ids, and the per-tet envelope coefficients */

/* History planes of a particle set: one device array [FEMPIC_DS_PLANES][n]
 * (plane-major, particle index fastest), f64 for an FP64-form env and f32
 * (f32 = 1) for a mixed-form env, owned by the caller:
 *   FEMPIC_DS_VH + 3*i + a     v^{n-1-i} along axis a, i = 0, 1, 2
 *   FEMPIC_DS_F  + 12*l + c    envelope sample of level n-1-l, l = 0, 1:
 *                              c = 0..2 Re E~, 3..5 Im E~, 6..8 Re B~, 9..11 Im B~
 *   FEMPIC_DS_VN, FEMPIC_DS_U  per-step scratch (new velocity, AB4 velocity)
 * Zero-initialised or not, it is filled by the first step (start = 1). */
#define FEMPIC_DS_VH 0
#define FEMPIC_DS_F 9
#define FEMPIC_DS_VN 33
#define FEMPIC_DS_U 36
#define FEMPIC_DS_PLANES 39

typedef struct {
  int64_t n;                 /* particles (same as the particle set) */
  void* planes;              /* device [FEMPIC_DS_PLANES][n], f64 or f32 */
  int32_t f32;               /* 1: f32 planes (mixed-form env), 0: f64 (FP64-form env) */
} fempic_downshift_history;

/* Build the gather tables (FP64 barycentric geometry, tet edges and faces)
 * from the same mesh description the env was created from, upload them to
 * the current device and allocate the per-tet coefficient buffer (20 f64 per
 * tet).  Errors: EINVAL, EMESH, ENOMEM, ECUDA.  Synchronizes the device. */
int fempic_downshift_create(const fempic_mesh_desc* mesh, fempic_downshift** out);

/* Host only, no GPU work: the weights of the step [t, t + dt] at carrier
 * frequency omega0, w_out[24] = {M^r[3], M^i[3], L^r[3][3], L^i[3][3]}
 * (row-major L[j][k]), for the basis on the node times t - k dt, k = 0, 1, 2.
 * Computed from the exact moments int_0^1 x^m e^{j theta x} dx, theta =
 * omega0 dt (power series for |theta| <= 1, recurrence above).
 * Errors: EINVAL (NULL, non-finite, dt <= 0). */
int fempic_downshift_weights(double t, double dt, double omega0, double* w_out);

/* One downshifted step from t to t + dt of every particle with tet >= 0, on
 * an env created from the mesh of ds: with FEMPIC_FP64, f64 velocities and
 * history and complex128 DoFs; with FEMPIC_MIXED or FEMPIC_MIXED_Q24, f32
 * velocities and history and complex64 DoFs (the per-tet coefficients are
 * built in FP64 and rounded once; samples, rule and AB4 in FP32).  Envelope
 * samples at r^n (Whitney sums of envl's DoFs times envl->amp = a(t), built
 * per tet as the affine form E~ = E0 + d x W, B~ = B0 + beta d), the
 * velocity rule, the AB4 segment tracked and deposited into the env's dG
 * (added to, not cleared), the history shifted.  start = 1 fills the history
 * with this step's own values first (constant extrapolation backwards).
 * Velocities are v^n on entry and v^{n+1} on exit (not half steps).
 * Particles with tet < 0 keep their state.  The per-tet coefficients live in
 * ds, so steps of one ds that overlap on the GPU (different streams) race;
 * give each concurrent particle set its own ds.  Errors: EINVAL (NULL,
 * sizes, species, scalars, a history of the other form), ECUDA, and any
 * error of the env's step.  Every argument is checked on the host before
 * the first launch, so an EINVAL leaves the particles and the history
 * untouched (a history whose f32 flag does not match the env's form is an
 * EINVAL too). */
int fempic_push_step_downshift(fempic_env* env, fempic_downshift* ds, const fempic_particles* p,
                               const fempic_downshift_history* hist, const fempic_envelope* envl,
                               double omega0, double t, double dt, int32_t start, void* stream);

/* Carry a history through a particle sort (the paper keeps particles in no
 * order; this keeps the downshifted step's history with its particles when
 * the set is re-sorted by tet for coalescing): for the planes that outlive a
 * step (FEMPIC_DS_VH .. FEMPIC_DS_VN - 1), out[k][q] = in[k][perm[q]], with
 * perm the permutation fempic_sort_perm returned for the same sort (perm[q] =
 * the index before the sort of particle q; a permutation of [0, n), device
 * int32 [n]).  in and out must not overlap.  Stream-ordered.  Errors:
 * EINVAL, ECUDA. */
int fempic_downshift_permute(const fempic_downshift_history* in, const fempic_downshift_history* out,
                             const int32_t* perm, void* stream);

const char* fempic_downshift_last_error(void);
void fempic_downshift_destroy(fempic_downshift* ds);

/* Debug build support (no counterpart in the paper).  In the debug build
 * (libfempic_env_debug.so, FEMPIC_BOUNDS_CHECK) the per-tet field pass of
 * fempic_push_step_downshift checks every edge and face id it reads from this
 * handle's tables before it addresses e_tilde / b_tilde; an out-of-range id
 * is skipped (that DoF reads as zero) and counted in the env's bounds
 * counter, so the next fempic_error_count on that env returns
 * FEMPIC_EBOUNDS.  This call overwrites one entry of this handle's device
 * tables so that the checks can be exercised:
 *   FEMPIC_TABLE_EDGE  index = 6 tet + local edge (edge ids, [nt][6]);
 *   FEMPIC_TABLE_FACE  index = 4 tet + local face (face ids, [nt][4]).
 * The release build refuses it (FEMPIC_EINVAL), so a corrupted table never
 * meets unchecked loads.  Synchronous.  Errors: EINVAL, ECUDA. */
int fempic_downshift_debug_set_table(fempic_downshift* ds, int32_t table, int64_t index, int32_t value);

#ifdef __cplusplus
}
#endif

#endif /* FEMPIC_DOWNSHIFT_H */
