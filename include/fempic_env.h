/*
 * fempic_env.h -- C ABI of the GB300 (sm_103a) particle hot path of the
 * envelope-tracking EM-FEMPIC method (Ramachandran et al., "An Envelope
 * Tracking Approach for Particle in Cell Simulations").
 *
 * One particle step, per particle, in order:
 *   (a) locate   carry the particle's tet; initial location = smallest-id tet
 *                whose four barycentrics are all >= 0;
 *   (b) gather   E~(r) = sum_e e~_e W1_e(r), B~(r) = sum_f b~_f W2_f(r)
 *                (Sec. III-A, Whitney expansion of the envelope fields);
 *   (c) carrier  E = Re{a(t) e^{j omega0 t} E~}, B = Re{a(t) e^{j omega0 t} B~}
 *                (Sec. III, envelope ansatz; Sec. III-D, Lorentz force with the
 *                fast carrier restored analytically);
 *   (d) push     Boris leapfrog, fields at (r^n, t_n), non-relativistic
 *                (Sec. III-D);
 *   (e) track    split r^n -> r^{n+1} at face crossings; reflecting (or
 *                absorbing) axis-aligned walls;
 *   (f) deposit  exact W1-tested path integral per in-tet segment,
 *                g_ij = q w (l_i(a) l_j(b) - l_j(a) l_i(b)), accumulated into
 *                the edge array dG (Sec. II eq. g_def; Sec. III-D eq.
 *                G_integral split into fine steps), and mapped into the
 *                envelope frame e^{-j omega0 t} G for the field solve
 *                (Sec. III-A, forcing term of eq. maxwell_semi).
 *
 * Conventions shared by every entry point
 *  - Mesh numbering: tet nodes are sorted by global id; edges [Ne][2] and
 *    faces [Nf][3] are numbered lexicographically by their sorted node tuples.
 *    Local edge e of a tet joins sorted local nodes (0,1),(0,2),(0,3),(1,2),
 *    (1,3),(2,3); local face k is opposite local node k.  Edge orientation is
 *    low -> high node id; face orientation (x_j - x_i) x (x_k - x_i), i<j<k.
 *  - Device pointers are CUDA global-memory pointers on the current device;
 *    host pointers are plain CPU memory.  Each field says which.
 *  - All calls taking a stream are asynchronous and stream-ordered on that
 *    cudaStream_t (passed as void*; NULL = legacy default stream) unless the
 *    comment says the call synchronizes.
 *  - Return value: FEMPIC_OK (0) or a negative FEMPIC_E* code; the message of
 *    the last failure on the calling thread is fempic_last_error().  No entry
 *    point traps or asserts on the device: bad particles get a status code.
 */
#ifndef FEMPIC_ENV_H
#define FEMPIC_ENV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define FEMPIC_OK 0
#define FEMPIC_EINVAL (-1)   /* bad argument (NULL, size, dtype/precision mismatch) */
#define FEMPIC_ECUDA (-2)    /* a CUDA runtime call failed */
#define FEMPIC_EMESH (-3)    /* degenerate (zero-volume) or non-conforming mesh */
#define FEMPIC_ENOMEM (-4)   /* host or device allocation failed */
#define FEMPIC_EINCOMPLETE (-5) /* a step did not finish all its particles (fempic_error_count) */
#define FEMPIC_EBOUNDS (-6)  /* debug build: a mesh-table index was out of range (fempic_error_count) */

/* ---- precision forms ---- */
#define FEMPIC_FP64 0   /* every step in FP64; velocities f64, DoFs complex128 */
#define FEMPIC_MIXED 1  /* gather, carrier product and push in FP32 (velocities f32,
                           DoFs complex64); positions and the position update in
                           FP64; the deposit, the barycentrics of tracking, the exit
                           parameter and the crossing barycentrics at FP64 accuracy
                           (exact products and double-float, 48-bit significands)
                           with FP64 crossing points and FP64 edge accumulation */
#define FEMPIC_MIXED_Q24 2 /* as FEMPIC_MIXED, but tracking and deposit on 24-bit
                           integer barycentrics: exit parameter in FP32, deposit
                           exact in int64 at a resolution of 2^-24 of a tet (charge
                           conserved exactly at that resolution) */

/* ---- per-particle status (uint8) ---- */
#define FEMPIC_P_OK 0
#define FEMPIC_P_CAP 1        /* more than max_crossings face crossings in one step */
#define FEMPIC_P_ABSORBED 2   /* left through a wall in absorb mode (or a non axis-aligned boundary) */
#define FEMPIC_P_NONFINITE 3  /* the push produced a non-finite velocity or position */
#define FEMPIC_P_LOST 4       /* no containing tet, or tet id out of range */
/* A frozen particle keeps its last tet T as tet = -2 - T; tet = -1 = no tet.
 * Particles with tet < 0 are skipped by every step. */

/* ---- wall modes ---- */
#define FEMPIC_WALL_REFLECT 0
#define FEMPIC_WALL_ABSORB 1

typedef struct fempic_env fempic_env;   /* opaque; owns derived mesh tables,
                                           accumulators and scratch on the device */

typedef struct {
  int64_t n_nodes;
  int64_t n_tets;
  const double* nodes_xyz;   /* host [n_nodes][3], copied at create */
  const int32_t* tet_nodes;  /* host [n_tets][4], any node order, copied at create */
  double bbox_lo[3];         /* axis-aligned walls: boundary faces lying in one of */
  double bbox_hi[3];         /* these six planes reflect (or absorb) particles     */
} fempic_mesh_desc;

typedef struct {
  int32_t precision;         /* FEMPIC_FP64, FEMPIC_MIXED or FEMPIC_MIXED_Q24 */
  int32_t max_crossings;     /* face crossings allowed per particle per step, 0 .. 2^20 */
  int32_t wall_mode;         /* FEMPIC_WALL_REFLECT or FEMPIC_WALL_ABSORB */
  int32_t reserved;          /* must be 0 */
} fempic_options;

typedef struct {
  int64_t n;                 /* number of particles */
  double* x;                 /* device f64 [n] positions (m) */
  double* y;
  double* z;
  void* vx;                  /* device velocities (m/s): f64 [n] (FP64 form) or f32 [n] (mixed forms) */
  void* vy;
  void* vz;
  int32_t* tet;              /* device i32 [n] current tet (see status convention) */
  uint8_t* status;           /* device u8 [n] FEMPIC_P_* */
  int32_t* n_cross;          /* device i32 [n] cumulative crossings, or NULL */
  int32_t n_species;         /* 1 .. 8 contiguous species ranges */
  const int64_t* species_begin; /* host [n_species+1], species s = [begin[s], begin[s+1]) */
  const double* q;           /* host [n_species] charge per physical particle (C) */
  const double* m;           /* host [n_species] mass (kg) */
  const double* w;           /* host [n_species] macro-particle weight */
} fempic_particles;

typedef struct {
  const void* e_tilde;       /* device complex [Ne] edge DoFs (interleaved re,im):
                                complex128 (FP64 form) or complex64 (mixed forms) */
  const void* b_tilde;       /* device complex [Nf] face DoFs, same dtype */
  double amp;                /* host scalar: slow envelope amplitude a(t) at this step */
} fempic_envelope;

/* Envelope interpolated in time from three DoF levels (Sec. III-D, the
 * simpler scheme that interpolates the downshifted fields to the fine step;
 * Sec. III-A, second-order Lagrange representation of the field
 * coefficients in time over [t_{n-1}, t_{n+1}]).  The envelope at t is
 * sum_k weight[k] level_k and the field is Re{amp e^{j omega0 t} (that sum)},
 * the carrier taken at t.  Level k is the envelope at tau_k = t_{n-1+k}, and
 * weight[k] is the second-order Lagrange basis function of tau_k evaluated
 * at t (fempic_lagrange3 computes it). */
typedef struct {
  const void* e_tilde[3];    /* device complex [Ne] edge DoFs of levels n-1, n, n+1, dtype as in
                                fempic_envelope */
  const void* b_tilde[3];    /* device complex [Nf] face DoFs of the same levels */
  double weight[3];          /* host: N_k(t) of each level */
  double amp;                /* host scalar: a(t) */
} fempic_envelope3;

typedef struct {
  int64_t n;                 /* number of particles (same as the particle set) */
  double* rx;                /* device f64 [n] adjoint of the positions */
  double* ry;
  double* rz;
  void* vx;                  /* device [n] adjoint of the velocities: f64 (FP64 form) or f32 (mixed) */
  void* vy;
  void* vz;
} fempic_adjoint;

/* Derive the mesh tables (sorted tet nodes, edges, faces, neighbours, wall
 * codes, FP64 barycentric geometry, point-location grid) on the host and
 * upload them to the current device; allocate the edge accumulators dG and
 * G_cum (zeroed).  Mesh: Sec. III-A / App. A sets N, E, F, T.
 * Errors: EINVAL (NULL, sizes, options), EMESH (zero-volume tet, a face in
 * more than two tets), ENOMEM, ECUDA.  Synchronizes the device. */
int fempic_env_create(const fempic_mesh_desc* mesh, const fempic_options* opts, fempic_env** out);

/* Sizes and tables of the derived numbering (host outputs; any may be NULL).
 * counts4 = {n_nodes, n_edges, n_faces, n_tets}.  tet_nbr: neighbour tet
 * across local face k, or a wall code -1-(2*axis+side) (side 0 = lo, 1 = hi),
 * or -7 for a boundary face off the bbox planes. */
int fempic_env_query(const fempic_env* env, int64_t* counts4, int32_t* tet_nodes /*[Nt][4]*/,
                     int32_t* edge_nodes /*[Ne][2]*/, int32_t* face_nodes /*[Nf][3]*/,
                     int32_t* tet_edges /*[Nt][6]*/, int32_t* tet_faces /*[Nt][4]*/,
                     int32_t* tet_nbr /*[Nt][4]*/);

/* (a) Initial location: tet[p] = smallest-id tet with all barycentrics >= 0
 * (FP64, fixed operation order), else tet = -1 and status = FEMPIC_P_LOST;
 * status = FEMPIC_P_OK for located particles.  Reads x, y, z; writes tet and
 * status.  Errors: EINVAL, ECUDA. */
int fempic_locate(fempic_env* env, const fempic_particles* p, void* stream);

/* (b)-(f) One fused particle step from t to t + dt for every particle with
 * tet >= 0: gather, carrier restore c = amp e^{j omega0 t} (phase and c in
 * FP64 on the host), Boris push, face tracking, and deposit of the path
 * integral into the env's dG accumulator (added to, not cleared).  Updates
 * x, y, z, v, tet, status and n_cross in place.  Velocities are v^{n-1/2} on
 * entry and v^{n+1/2} on exit.  Errors: EINVAL (precision/dtype mismatch,
 * species ranges), ECUDA. */
int fempic_push_step(fempic_env* env, const fempic_particles* p, const fempic_envelope* envl,
                     double omega0, double t, double dt, void* stream);

/* The step of fempic_push_step with the envelope interpolated from three
 * levels (fempic_envelope3): only the per-tet field construction reads the
 * extra levels; the particle work is the same.  Errors: as fempic_push_step,
 * and EINVAL for a NULL level or a non-finite weight. */
int fempic_push_step3(fempic_env* env, const fempic_particles* p, const fempic_envelope3* envl,
                      double omega0, double t, double dt, void* stream);

/* Second-order Lagrange weights (Sec. III-A): w_out[k] = prod_{j != k}
 * (t - tau[j]) / (tau[k] - tau[j]) for three distinct level times tau[3];
 * host only, no GPU work.  Errors: EINVAL (NULL, non-finite or repeated
 * times). */
int fempic_lagrange3(const double* tau, double t, double* w_out);

/* Finalize the deposit of one step (Sec. III-D, eq. G_integral; forcing term
 * e^{-j omega0 t} G of Sec. III-A): G_cum += dG; then, when non-NULL,
 *   dG_out    <- dG                               (device f64 [Ne])
 *   G_cum_out <- G_cum                            (device f64 [Ne])
 *   G_env_out <- e^{-j omega0 t_next} G_cum       (device complex128 [Ne])
 * and dG is zeroed.  Errors: EINVAL, ECUDA. */
int fempic_deposit(fempic_env* env, double omega0, double t_next, double* dG_out, double* G_cum_out,
                   void* G_env_out, void* stream);

/* The two halves of fempic_deposit for a run whose particles are sharded
 * over several processes (each GPU holds the whole mesh and DoFs and a range
 * of the particles; the only coupling is the sum of the edge deposit, Sec.
 * III-D eq. G_integral, over the shards):
 *   fempic_deposit_local  finalizes this process's step deposit into dG_out
 *                         (device f64 [Ne]) and clears the accumulator,
 *                         leaving G_cum unchanged;
 *   fempic_accumulate     adds a step deposit dG (device f64 [Ne], the
 *                         all-reduced sum of every shard's dG_out) to G_cum
 *                         and writes, when non-NULL, G_cum_out and
 *                         G_env_out = e^{-j omega0 t_next} G_cum as
 *                         fempic_deposit does.
 * fempic_deposit on one process equals fempic_deposit_local followed by
 * fempic_accumulate of that dG_out.  Stream-ordered.  Errors: EINVAL, ECUDA. */
int fempic_deposit_local(fempic_env* env, double* dG_out, void* stream);
int fempic_accumulate(fempic_env* env, double omega0, double t_next, const double* dG, double* G_cum_out,
                      void* G_env_out, void* stream);

/* Switch the deposit (f) of later push steps on (enable != 0, the default)
 * or off.  Off, a step still gathers, pushes and tracks every particle
 * exactly as with the deposit on, but adds nothing to dG: for callers that
 * need only the trajectories, such as the gradient of a loss that does not
 * depend on the deposited charge (the paper's method always deposits; this
 * switch has no counterpart there).  Host only.  Errors: EINVAL. */
int fempic_set_deposit(fempic_env* env, int32_t enable);

/* Zero dG and G_cum (start of a run).  Errors: ECUDA. */
int fempic_reset_deposit(fempic_env* env, void* stream);

/* Whitney-0 nodal charge rho_n = sum_p q w lambda_n(r_p) (Sec. III-B,
 * discrete Gauss law: charge on nodes) over particles with a known tet,
 * written to rho (device f64 [Nn], overwritten).  Used with the edge
 * divergence to check charge conservation D^T G_cum = rho^n - rho^0.
 * Errors: EINVAL, ECUDA. */
int fempic_nodal_charge(fempic_env* env, const fempic_particles* p, double* rho, void* stream);

/* Host-side counters accumulated by push_step since create:
 * out4 = {face crossings, particles frozen (any non-OK status), steps,
 * staging waits that gave up}.  The last one counts CTAs of the staged push
 * kernel whose bounded wait (about 1 s) for a bulk copy expired; they stop
 * early, so any non-zero value means that step's results are incomplete.
 * Synchronizes the stream.  Errors: EINVAL, ECUDA. */
int fempic_stats(fempic_env* env, int64_t* out4, void* stream);

/* Error report of the steps since the last call (or since create), for
 * callers of the asynchronous push step (Sec. III-D particle step; the paper
 * has no error path).  Synchronizes `stream`, then sets *n_bad to the number
 * of particles those steps froze (status CAP, ABSORBED, NONFINITE or LOST)
 * and returns FEMPIC_OK, or FEMPIC_EINCOMPLETE when, in one of those steps, a
 * CTA of the staged mixed push gave up its bounded wait (about 1 s) for a
 * bulk copy: the particles of its remaining tiles were then not advanced and
 * their deposit is missing, so the step must be redone from a saved state.
 * In the debug build it returns FEMPIC_EBOUNDS when a mesh-table index out of
 * range was skipped (fempic_debug_set_table; the downshifted step's own
 * tables, fempic_downshift_debug_set_table, count here too).  fempic_stats keeps the
 * cumulative counters.  Errors: EINVAL, ECUDA, EINCOMPLETE, EBOUNDS. */
int fempic_error_count(fempic_env* env, int64_t* n_bad, void* stream);

/* Test support for the bounded waits (no counterpart in the paper): in the
 * next push step only, CTA `cta` of the staged mixed push kernel (if that
 * launch has such a CTA) waits, after its first tile's copies have landed, on
 * a barrier that no copy completes, with every bounded wait of that launch
 * limited to limit_ns (1e3 .. 1e9).  The wait runs out, the CTA drains its
 * copies in flight and stops, and fempic_error_count reports
 * FEMPIC_EINCOMPLETE: the give-up path runs without any device fault.
 * Host only.  Errors: EINVAL. */
int fempic_debug_stall(fempic_env* env, int32_t cta, int64_t limit_ns);

/* Debug build support (no counterpart in the paper).  The library's debug
 * build, libfempic_env_debug.so (compiled with FEMPIC_BOUNDS_CHECK), checks
 * every index read from a mesh table against its range before it addresses
 * memory; a bad index is skipped (a DoF reads as zero, a deposit term is
 * dropped, a walking particle freezes with status LOST) and counted, and the
 * next fempic_error_count returns FEMPIC_EBOUNDS.  This call overwrites one
 * entry of a device mesh table so that the checks can be exercised:
 *   FEMPIC_TABLE_NEIGHBOUR  index = 4 tet + local face (the neighbour table
 *                           and its copy in the tet record);
 *   FEMPIC_TABLE_EDGE       index = 6 tet + local edge (the edge-id table).
 * FEMPIC_TABLE_FACE (index = 4 tet + local face, the face-id table) is
 * accepted by fempic_downshift_debug_set_table only.
 * The release build refuses it (FEMPIC_EINVAL), so a corrupted table never
 * meets unchecked loads.  Synchronous.  Errors: EINVAL, ECUDA. */
#define FEMPIC_TABLE_NEIGHBOUR 0
#define FEMPIC_TABLE_EDGE 1
#define FEMPIC_TABLE_FACE 2
int fempic_debug_set_table(fempic_env* env, int32_t table, int64_t index, int32_t value);

/* Deposited-current term of the loss for the adjoint steps (the paper has no
 * adjoint; this differentiates the per-segment deposit g_ij of Sec. II eq.
 * g_def as the push step applies it): u (device f64 [Ne], read now, not
 * kept) weights each edge's deposit, and every later
 * fempic_push_step_adjoint adds the gradient of sum_e u_e dG_e over its
 * step, dG the step's edge deposit for the species' q w.  The gradient
 * follows the step's FP64 face walk (the mixed forms' walk agrees with it
 * except where a path grazes an edge or vertex within the FP32 filter's
 * margin).  Per tet the kernel stores alpha = sum_j u_{0j} grad l_j and
 * beta = sum_{i<j} u_{ij} grad l_i x grad l_j (48 B, allocated on first
 * use).  u == NULL turns the term off.  Stream-ordered.  Errors: EINVAL,
 * ECUDA. */
int fempic_adjoint_current_weights(fempic_env* env, const double* u, void* stream);

/* Reverse mode of one fempic_push_step (gradients of a loss of the particle
 * state after some steps, with respect to the envelope DoFs and the initial
 * phase space; the paper has no adjoint, this differentiates its particle
 * step: gather, carrier, Boris, position update and wall mirrors, Sec. III-D).
 * `before` is the particle state the forward step started from and `after`
 * the state it produced (only velocities and statuses of `after` are read:
 * a velocity component with the opposite sign marks a wall mirror, a
 * non-OK status a freeze).  On entry adj holds the adjoint of `after`; on
 * exit the adjoint of `before`.  The derivative is that of the piecewise
 * smooth map for the tet sequence the forward step took.  Particles frozen
 * during the step get a zero adjoint (plus, with current weights set, the
 * gradient of the charge they moved before freezing).  When
 * fempic_adjoint_current_weights has set weights u, the loss also holds
 * sum_e u_e dG_e of this step's deposit, and its gradient is added.  e_grad (complex128 [Ne]) and b_grad
 * (complex128 [Nf]) accumulate dL/dRe + j dL/dIm of the DoFs (added to, in
 * FP64).  The mixed form differentiates its FP32 push in FP32 and keeps the
 * position adjoint and the DoF gradients in FP64.  Stream-ordered; the
 * field pre-pass of this step is recomputed.  Errors: EINVAL, ECUDA. */
int fempic_push_step_adjoint(fempic_env* env, const fempic_particles* before, const fempic_particles* after,
                             const fempic_envelope* envl, double omega0, double t, double dt,
                             const fempic_adjoint* adj, void* e_grad, void* b_grad, void* stream);

/* Total kinetic energy sum_p 1/2 m w |v|^2 over particles with tet >= 0,
 * written to *ke (device f64 scalar, overwritten).  When seed is non-NULL it
 * also receives the adjoint of that loss: vbar = m w v, rbar = 0 (0 for
 * particles without a tet).  Stream-ordered.  Errors: EINVAL, ECUDA. */
int fempic_kinetic_energy(fempic_env* env, const fempic_particles* p, double* ke, const fempic_adjoint* seed,
                          void* stream);

/* Keep the particle SoA ordered for coalesced, tet-local access (the
 * particle state of Sec. III-D in a GPU layout; no counterpart in the
 * paper's method): out = in permuted so that each species range stays in
 * place and, inside it, particles are ordered by tet id, with particles of
 * tet < 0 (frozen or unlocated) last.  Order inside one tet is unspecified.
 * in and out are two caller-owned particle sets with the same n, velocity
 * dtype and species table, and must not overlap; n_cross may be NULL in both
 * (else in both).  The counting scratch (one int32 counter per (species,
 * tet) key) is owned by the env and grown on demand.  Stream-ordered.
 * Errors: EINVAL (mismatch), ENOMEM, ECUDA. */
int fempic_sort(fempic_env* env, const fempic_particles* in, const fempic_particles* out, void* stream);

/* fempic_sort that also writes perm[q] = the index in `in` of the particle
 * placed at position q of `out` (device int32 [n], caller owned), so that
 * per-particle data kept elsewhere (an adjoint state) can follow the sort.
 * Errors: as fempic_sort, and EINVAL for a NULL perm. */
int fempic_sort_perm(fempic_env* env, const fempic_particles* in, const fempic_particles* out, int32_t* perm,
                     void* stream);

/* Carry an adjoint state back across a sort (the transpose of the
 * permutation fempic_sort_perm applied to the particles): out[perm[q]] =
 * in[q] for rbar (f64) and vbar (the env's velocity dtype).  in and out are
 * caller-owned device arrays of the same n that must not overlap; perm must
 * be a permutation of 0..n-1 (entries outside that range are skipped).
 * Stream-ordered.  Errors: EINVAL, ECUDA. */
int fempic_adjoint_unpermute(fempic_env* env, const fempic_adjoint* in, const fempic_adjoint* out,
                             const int32_t* perm, void* stream);

/* Same sort as fempic_sort, for callers that must not allocate device
 * memory once they are running (the paper has no counterpart; this is an
 * integration entry point).  Examples: an application whose device memory is
 * all handed out up front to its own pool allocator, so a cudaMalloc would
 * fail or fragment that pool; a time-critical loop that cannot afford the
 * device-wide synchronization cudaFree implies.  fempic_sort grows its
 * counting scratch with cudaMalloc/cudaFree on demand; this entry point
 * instead uses a fixed scratch area compiled into the library (about 16 MB
 * of device memory that every GPU which loads the library keeps until the
 * process exits), and calls no allocating routine.
 *   Limit: n_species * (n_tets + 1) <= FEMPIC_SORT_NOALLOC_MAX_KEYS, else
 *   FEMPIC_EINVAL with a message; n < 2^31.
 *   Set-up: the first call on each device (with that device current) looks
 *   up the scratch area's device address once; make that first call before
 *   any stream capture.
 *   Sharing: all calls in the process use the same scratch area, which keeps
 *   the contents of the last call; each call clears what it needs.  Calls
 *   whose work overlaps on the GPU (different streams, or different threads
 *   without ordering) race on that area and give wrong results: order them.
 * in, out, env, ordering and errors are as for fempic_sort; this call records
 * no per-kernel timing. */
#define FEMPIC_SORT_NOALLOC_MAX_KEYS (1 << 21)
int fempic_sort_noalloc(fempic_env* env, const fempic_particles* in, const fempic_particles* out,
                        void* stream);

/* Kernel ids of the per-kernel timing below. */
#define FEMPIC_K_LOCATE 0
#define FEMPIC_K_FIELD 1      /* per-tet carrier restore + affine field coefficients */
#define FEMPIC_K_PUSH 2       /* fused gather/push/track/deposit */
#define FEMPIC_K_FINALIZE 3   /* deposit finalize */
#define FEMPIC_K_CHARGE 4     /* nodal charge */
#define FEMPIC_K_SORT 5       /* particle sort by tet */
#define FEMPIC_K_CROSS 6      /* crossing pass; its bracket lies inside FEMPIC_K_PUSH's */
#define FEMPIC_K_ADJOINT 7    /* adjoint step: field rebuild, particle adjoint, field adjoint */
#define FEMPIC_K_COUNT 8

/* Measurement support (no counterpart in the paper): while enabled, every
 * kernel the env launches is bracketed by two CUDA events recorded on its
 * launch stream.  enable != 0 clears earlier records and starts recording;
 * 0 stops.  At most 65536 launches are recorded per enable.  Errors: EINVAL. */
int fempic_profile_enable(fempic_env* env, int32_t enable);

/* Per kernel id, since the last enable: summed bracket durations in ms
 * (ms_out[FEMPIC_K_COUNT]), the number of brackets, one per library call
 * (calls_out[FEMPIC_K_COUNT]), and the number of kernels launched inside
 * them (kernels_out[FEMPIC_K_COUNT]; a nested bracket's kernels count under
 * its own id only, so the sum over ids is the number of kernel launches).
 * Synchronizes on the recorded events.  Errors: EINVAL, ECUDA. */
int fempic_profile_read(fempic_env* env, double* ms_out, int64_t* calls_out, int64_t* kernels_out);

/* Measurement support (no counterpart in the paper): the FP64 fused
 * multiply-add rate of the current device in lane operations per second,
 * from one timed launch of independent FMA chains on every SM (after one
 * untimed launch), written to *lane_ops_per_s (host).  It is the ceiling of
 * the FP64 form, whose step is FP64-pipe bound on GB300.  Allocates 8 bytes
 * of device memory for the duration of the call; synchronizes `stream`.
 * Errors: EINVAL, ECUDA. */
int fempic_measure_fp64_rate(double* lane_ops_per_s, void* stream);

/* Message of the last failure on the calling thread ("" if none). */
const char* fempic_last_error(void);

/* Free everything the env owns.  Safe on NULL. */
void fempic_env_destroy(fempic_env* env);

#ifdef __cplusplus
}
#endif
#endif /* FEMPIC_ENV_H */
