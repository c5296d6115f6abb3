/*
 * fempic_oracle.c -- plain, slow, serial FP64 CPU oracle of the
 * envelope-tracking FEMPIC particle step (Ramachandran et al.,
 * "An Envelope Tracking Approach for Particle in Cell Simulations").
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code, header,
 * table or constant with the CUDA library: it derives its own mesh tables
 * from the raw node/tet arrays.
 *
 * What one particle step computes, per particle, in this order (Sec. III):
 *
 *  (a) locate   the particle's tet is carried in the particle state; the
 *               initial tet is the smallest-id tet whose four barycentrics
 *               are all >= 0 (or_locate*).
 *  (b) gather   E~(r) = sum_e e~_e W1_e(r), B~(r) = sum_f b~_f W2_f(r)
 *               (Sec. III-A, Whitney expansion of the envelope fields), with
 *               the textbook Whitney forms on barycentrics lambda:
 *                 W1_ij  = lambda_i grad(lambda_j) - lambda_j grad(lambda_i)
 *                 W2_ijl = 2 (lambda_i gl_j x gl_l + lambda_j gl_l x gl_i
 *                             + lambda_l gl_i x gl_j),  gl = grad lambda.
 *               Tet nodes are sorted by global id, so every local edge/face
 *               orientation equals the global one (edge low->high id, face
 *               normal (x_j - x_i) x (x_l - x_i) for i<j<l).
 *  (c) carrier  E = Re{c E~}, B = Re{c B~}, c = a(t) e^{j omega0 t}
 *               (Sec. III-D, Lorentz force with the fast carrier restored).
 *  (d) push     Boris leapfrog with fields sampled at (r^n, t_n); initial
 *               velocities are v^{-1/2}; non-relativistic (Sec. III-D).
 *  (e) track    the straight segment r^n -> r^{n+1} is split at every face
 *               crossing; reflecting axis-aligned walls mirror the remaining
 *               displacement and the velocity component.
 *  (f) deposit  per segment a->b inside one tet, the exact W1-tested path
 *               integral g_ij = q w (lambda_i(a) lambda_j(b) - lambda_j(a)
 *               lambda_i(b)) is added to dG of that edge (Sec. II eq. g_def,
 *               Sec. III-D eq. G_integral and its fine-step split).
 *
 * Fixed operation order (no FMA: build with -ffp-contract=off).  Sums are
 * evaluated left to right as written.
 *   geometry  e_k = x_k - x_0 (k=1..3); c1 = e2 x e3, c2 = e3 x e1,
 *             c3 = e1 x e2; (u x w)_x = u_y w_z - u_z w_y (cyclic);
 *             det = (e1x c1x + e1y c1y) + e1z c1z;  gl_k = c_k / det (per
 *             component, k=1..3);  gl_0 = -((gl_1 + gl_2) + gl_3).
 *   lambda    d = r - x_0;  lambda_k = (gl_kx dx + gl_ky dy) + gl_kz dz
 *             (k=1..3);  lambda_0 = ((1 - lambda_1) - lambda_2) - lambda_3.
 *   gather    W1 per component (lambda_i gl_j) - (lambda_j gl_i); field
 *             sums accumulate from 0 in local edge order (01,02,03,12,13,23)
 *             and local face order (face k opposite node k); for the W2 of
 *             face (i,j,l): 2 * ((lambda_i c_jl + lambda_j c_li) + lambda_l
 *             c_ij) with c_jl = gl_j x gl_l etc.  Complex DoFs: real and
 *             imaginary parts accumulate separately.
 *   carrier   phi = omega0 * t; c = (amp*cos(phi), amp*sin(phi));
 *             E = (c_re E~_re) - (c_im E~_im) per component.
 *   Boris     k = ((q/m) dt) 0.5;  v- = v + k E;  tau = k B;
 *             t2 = (tau_x^2 + tau_y^2) + tau_z^2;  f = 2/(1 + t2);
 *             s = f tau;  v' = v- + (v- x tau);  v+ = v- + (v' x s);
 *             v_new = v+ + k E;  b = r + dt v_new.
 *   track     in tet T with lambda(a): lambda(b) from b's coordinates;
 *             candidate faces k != entry with lambda_k(b) < 0; for each,
 *             s_k = lambda_k(a) / (lambda_k(a) - lambda_k(b)), s_k < 0 -> 0;
 *             the exit face is the strict argmin (ties: lowest k).  None:
 *             deposit a->b and stop.  Else p = a + s (b - a) per component;
 *             lambda_i(p) = lambda_i(a) + s (lambda_i(b) - lambda_i(a)) for
 *             i != k and lambda_k(p) = 0; deposit a->p; count the crossing;
 *             more than max_crossings crossings -> status CAP, frozen at p.
 *             Interior face: move to the neighbour T', whose lambda(p) takes
 *             the values of the shared nodes and 0 at its own opposite node;
 *             the entry face of T' is excluded.  Wall face: reflect mode
 *             mirrors b_axis <- (2 L) - b_axis, v_axis <- -v_axis and
 *             continues from p in T with the wall face as entry; absorb mode
 *             freezes the particle at p with status ABSORBED.
 *   deposit   for local edge (i,j): dG += (q w) * ((la_i lb_j) - (la_j lb_i)).
 *
 * Particle status: 0 OK, 1 CAP, 2 ABSORBED, 3 NONFINITE (push produced a
 * non-finite value: particle left unmoved), 4 LOST (no containing tet / tet
 * id out of range).  A frozen particle keeps its last tet T encoded as
 * tet = -2 - T; tet = -1 means no tet.  Particles with tet < 0 are skipped.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_CAP 1
#define OR_ABSORBED 2
#define OR_NONFINITE 3
#define OR_LOST 4

static const int LE[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
static const int LF[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

typedef struct {
  int64_t nn, nt, ne, nf;
  double *xyz;   /* [nn][3] */
  int32_t *tn;   /* [nt][4] sorted node ids */
  int32_t *en;   /* [ne][2] */
  int32_t *fn;   /* [nf][3] */
  int32_t *te;   /* [nt][6] */
  int32_t *tf;   /* [nt][4] */
  int32_t *nb;   /* [nt][4] neighbour tet, or wall code -1-(2*axis+side), -7 other boundary */
  double *gl;    /* [nt][4][3] barycentric gradients */
  double lo[3], hi[3];
  int gd[3];
  double ginv[3];
  int64_t *gstart; /* [ncell+1] */
  int32_t *gtet;
} omesh;

/* ------------------------------------------------------------------ utils */
static int cmp_i64(const void *a, const void *b) {
  int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
  return (x > y) - (x < y);
}
static int cmp_tri(const void *a, const void *b) {
  const int32_t *x = (const int32_t *)a, *y = (const int32_t *)b;
  for (int i = 0; i < 3; i++) {
    if (x[i] != y[i]) return (x[i] > y[i]) - (x[i] < y[i]);
  }
  return 0;
}
static void cross3(const double *u, const double *w, double *o) {
  o[0] = u[1] * w[2] - u[2] * w[1];
  o[1] = u[2] * w[0] - u[0] * w[2];
  o[2] = u[0] * w[1] - u[1] * w[0];
}
static int64_t find_i64(const int64_t *a, int64_t n, int64_t key) {
  int64_t lo = 0, hi = n - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (a[mid] == key) return mid;
    if (a[mid] < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}
static int64_t find_tri(const int32_t *a, int64_t n, const int32_t *key) {
  int64_t lo = 0, hi = n - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    int c = cmp_tri(a + 3 * mid, key);
    if (c == 0) return mid;
    if (c < 0) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

/* ---------------------------------------------------------- barycentrics */
void or_bary(const omesh *m, int32_t t, const double *r, double *lam) {
  const double *x0 = m->xyz + 3 * (int64_t)m->tn[4 * (int64_t)t];
  const double *g = m->gl + 12 * (int64_t)t;
  double dx = r[0] - x0[0], dy = r[1] - x0[1], dz = r[2] - x0[2];
  for (int k = 1; k < 4; k++)
    lam[k] = (g[3 * k] * dx + g[3 * k + 1] * dy) + g[3 * k + 2] * dz;
  lam[0] = ((1.0 - lam[1]) - lam[2]) - lam[3];
}

void or_grad_bary(const omesh *m, int32_t t, double *g12) {
  memcpy(g12, m->gl + 12 * (int64_t)t, 12 * sizeof(double));
}

/* ------------------------------------------------------------------ mesh */
static void free_mesh(omesh *m) {
  if (!m) return;
  free(m->xyz); free(m->tn); free(m->en); free(m->fn); free(m->te); free(m->tf);
  free(m->nb); free(m->gl); free(m->gstart); free(m->gtet);
  free(m);
}

static int cell_of(const omesh *m, int a, double x) {
  double f = floor((x - m->lo[a]) * m->ginv[a]);
  if (!(f >= 0.0)) return 0;                 /* also catches NaN */
  if (f > (double)(m->gd[a] - 1)) return m->gd[a] - 1;
  return (int)f;
}

/* Uniform bucket grid: every tet goes into all cells its bounding box
 * overlaps, using the same monotone cell_of() as the query, so every tet that
 * contains a point is listed in that point's cell.  Lists are ascending. */
static int build_grid(omesh *m) {
  double g = cbrt((double)m->nt / 6.0);
  int gd = (int)(g + 0.5);
  if (gd < 1) gd = 1;
  if (gd > 256) gd = 256;
  for (int a = 0; a < 3; a++) {
    m->gd[a] = gd;
    double ext = m->hi[a] - m->lo[a];
    m->ginv[a] = ext > 0.0 ? (double)gd / ext : 0.0;
  }
  int64_t ncell = (int64_t)gd * gd * gd;
  int64_t *cnt = calloc((size_t)ncell + 1, sizeof(int64_t));
  if (!cnt) return -1;
  for (int pass = 0; pass < 2; pass++) {
    for (int64_t t = 0; t < m->nt; t++) {
      int c0[3], c1[3];
      for (int a = 0; a < 3; a++) {
        double mn = INFINITY, mx = -INFINITY;
        for (int v = 0; v < 4; v++) {
          double x = m->xyz[3 * (int64_t)m->tn[4 * t + v] + a];
          if (x < mn) mn = x;
          if (x > mx) mx = x;
        }
        c0[a] = cell_of(m, a, mn);
        c1[a] = cell_of(m, a, mx);
      }
      for (int k = c0[2]; k <= c1[2]; k++)
        for (int j = c0[1]; j <= c1[1]; j++)
          for (int i = c0[0]; i <= c1[0]; i++) {
            int64_t c = i + (int64_t)gd * (j + (int64_t)gd * k);
            if (pass == 0) cnt[c + 1]++;
            else m->gtet[cnt[c]++] = (int32_t)t;
          }
    }
    if (pass == 0) {
      for (int64_t c = 0; c < ncell; c++) cnt[c + 1] += cnt[c];
      m->gstart = malloc(sizeof(int64_t) * (size_t)(ncell + 1));
      m->gtet = malloc(sizeof(int32_t) * (size_t)(cnt[ncell] > 0 ? cnt[ncell] : 1));
      if (!m->gstart || !m->gtet) { free(cnt); return -1; }
      memcpy(m->gstart, cnt, sizeof(int64_t) * (size_t)(ncell + 1));
    }
  }
  free(cnt);
  return 0;
}

/* Returns a mesh handle, or NULL with *err set: 1 bad input / allocation,
 * 2 degenerate tet (zero volume), 3 non-conforming (face in > 2 tets). */
void *or_mesh_create(int64_t nn, const double *xyz, int64_t nt, const int32_t *tets,
                     const double *lo, const double *hi, int32_t *err) {
  *err = 0;
  omesh *m = calloc(1, sizeof(omesh));
  if (!m || nn <= 0 || nt <= 0) { *err = 1; free(m); return NULL; }
  m->nn = nn; m->nt = nt;
  for (int a = 0; a < 3; a++) { m->lo[a] = lo[a]; m->hi[a] = hi[a]; }
  m->xyz = malloc(sizeof(double) * 3 * (size_t)nn);
  m->tn = malloc(sizeof(int32_t) * 4 * (size_t)nt);
  if (!m->xyz || !m->tn) { *err = 1; free_mesh(m); return NULL; }
  memcpy(m->xyz, xyz, sizeof(double) * 3 * (size_t)nn);
  for (int64_t t = 0; t < nt; t++) {
    int32_t v[4];
    for (int i = 0; i < 4; i++) {
      v[i] = tets[4 * t + i];
      if (v[i] < 0 || v[i] >= nn) { *err = 1; free_mesh(m); return NULL; }
    }
    for (int i = 1; i < 4; i++) {          /* insertion sort */
      int32_t x = v[i]; int j = i - 1;
      while (j >= 0 && v[j] > x) { v[j + 1] = v[j]; j--; }
      v[j + 1] = x;
    }
    for (int i = 0; i < 4; i++) m->tn[4 * t + i] = v[i];
  }
  /* edges: keys lo*nn + hi, sorted, unique */
  int64_t *ek = malloc(sizeof(int64_t) * 6 * (size_t)nt);
  if (!ek) { *err = 1; free_mesh(m); return NULL; }
  for (int64_t t = 0; t < nt; t++)
    for (int e = 0; e < 6; e++)
      ek[6 * t + e] = (int64_t)m->tn[4 * t + LE[e][0]] * nn + m->tn[4 * t + LE[e][1]];
  int64_t *eks = malloc(sizeof(int64_t) * 6 * (size_t)nt);
  if (!eks) { free(ek); *err = 1; free_mesh(m); return NULL; }
  memcpy(eks, ek, sizeof(int64_t) * 6 * (size_t)nt);
  qsort(eks, (size_t)(6 * nt), sizeof(int64_t), cmp_i64);
  int64_t ne = 0;
  for (int64_t i = 0; i < 6 * nt; i++)
    if (i == 0 || eks[i] != eks[i - 1]) eks[ne++] = eks[i];
  m->ne = ne;
  m->en = malloc(sizeof(int32_t) * 2 * (size_t)ne);
  m->te = malloc(sizeof(int32_t) * 6 * (size_t)nt);
  if (!m->en || !m->te) { free(ek); free(eks); *err = 1; free_mesh(m); return NULL; }
  for (int64_t e = 0; e < ne; e++) {
    m->en[2 * e] = (int32_t)(eks[e] / nn);
    m->en[2 * e + 1] = (int32_t)(eks[e] % nn);
  }
  for (int64_t i = 0; i < 6 * nt; i++) m->te[i] = (int32_t)find_i64(eks, ne, ek[i]);
  free(ek); free(eks);
  /* faces: sorted node triples, sorted lexicographically, unique */
  int32_t *fk = malloc(sizeof(int32_t) * 12 * (size_t)nt);
  int32_t *fks = malloc(sizeof(int32_t) * 12 * (size_t)nt);
  if (!fk || !fks) { free(fk); free(fks); *err = 1; free_mesh(m); return NULL; }
  for (int64_t t = 0; t < nt; t++)
    for (int f = 0; f < 4; f++)
      for (int i = 0; i < 3; i++) fk[12 * t + 3 * f + i] = m->tn[4 * t + LF[f][i]];
  memcpy(fks, fk, sizeof(int32_t) * 12 * (size_t)nt);
  qsort(fks, (size_t)(4 * nt), 3 * sizeof(int32_t), cmp_tri);
  int64_t nf = 0;
  for (int64_t i = 0; i < 4 * nt; i++)
    if (i == 0 || cmp_tri(fks + 3 * i, fks + 3 * (i - 1)) != 0) {
      memmove(fks + 3 * nf, fks + 3 * i, 3 * sizeof(int32_t));
      nf++;
    }
  m->nf = nf;
  m->fn = malloc(sizeof(int32_t) * 3 * (size_t)nf);
  m->tf = malloc(sizeof(int32_t) * 4 * (size_t)nt);
  if (!m->fn || !m->tf) { free(fk); free(fks); *err = 1; free_mesh(m); return NULL; }
  memcpy(m->fn, fks, sizeof(int32_t) * 3 * (size_t)nf);
  for (int64_t i = 0; i < 4 * nt; i++) m->tf[i] = (int32_t)find_tri(fks, nf, fk + 3 * i);
  free(fk); free(fks);
  /* neighbours through faces */
  int32_t *ft = malloc(sizeof(int32_t) * 2 * (size_t)nf);
  m->nb = malloc(sizeof(int32_t) * 4 * (size_t)nt);
  if (!ft || !m->nb) { free(ft); *err = 1; free_mesh(m); return NULL; }
  for (int64_t f = 0; f < 2 * nf; f++) ft[f] = -1;
  for (int64_t t = 0; t < nt; t++)
    for (int k = 0; k < 4; k++) {
      int64_t f = m->tf[4 * t + k];
      if (ft[2 * f] < 0) ft[2 * f] = (int32_t)t;
      else if (ft[2 * f + 1] < 0) ft[2 * f + 1] = (int32_t)t;
      else { free(ft); *err = 3; free_mesh(m); return NULL; }
    }
  for (int64_t t = 0; t < nt; t++)
    for (int k = 0; k < 4; k++) {
      int64_t f = m->tf[4 * t + k];
      int32_t o = ft[2 * f] == (int32_t)t ? ft[2 * f + 1] : ft[2 * f];
      if (o >= 0) { m->nb[4 * t + k] = o; continue; }
      int32_t code = -7;
      for (int a = 0; a < 3 && code == -7; a++)
        for (int s = 0; s < 2 && code == -7; s++) {
          double L = s ? hi[a] : lo[a];
          int on = 1;
          for (int i = 0; i < 3; i++)
            if (m->xyz[3 * (int64_t)m->fn[3 * f + i] + a] != L) on = 0;
          if (on) code = -1 - (2 * a + s);
        }
      m->nb[4 * t + k] = code;
    }
  free(ft);
  /* geometry */
  m->gl = malloc(sizeof(double) * 12 * (size_t)nt);
  if (!m->gl) { *err = 1; free_mesh(m); return NULL; }
  for (int64_t t = 0; t < nt; t++) {
    const double *x0 = m->xyz + 3 * (int64_t)m->tn[4 * t];
    double e[3][3], c[3][3];
    for (int k = 0; k < 3; k++) {
      const double *xk = m->xyz + 3 * (int64_t)m->tn[4 * t + k + 1];
      for (int a = 0; a < 3; a++) e[k][a] = xk[a] - x0[a];
    }
    cross3(e[1], e[2], c[0]);
    cross3(e[2], e[0], c[1]);
    cross3(e[0], e[1], c[2]);
    double det = (e[0][0] * c[0][0] + e[0][1] * c[0][1]) + e[0][2] * c[0][2];
    if (!(det != 0.0) || !isfinite(det)) { *err = 2; free_mesh(m); return NULL; }
    double *g = m->gl + 12 * t;
    for (int k = 0; k < 3; k++)
      for (int a = 0; a < 3; a++) g[3 * (k + 1) + a] = c[k][a] / det;
    for (int a = 0; a < 3; a++) g[a] = -((g[3 + a] + g[6 + a]) + g[9 + a]);
  }
  if (build_grid(m) != 0) { *err = 1; free_mesh(m); return NULL; }
  return m;
}

void or_mesh_destroy(void *h) { free_mesh((omesh *)h); }

void or_mesh_sizes(const void *h, int64_t *out4) {
  const omesh *m = (const omesh *)h;
  out4[0] = m->nn; out4[1] = m->ne; out4[2] = m->nf; out4[3] = m->nt;
}

void or_mesh_tables(const void *h, int32_t *tet_nodes, int32_t *edge_nodes, int32_t *face_nodes,
                    int32_t *tet_edges, int32_t *tet_faces, int32_t *tet_nbr) {
  const omesh *m = (const omesh *)h;
  if (tet_nodes) memcpy(tet_nodes, m->tn, sizeof(int32_t) * 4 * (size_t)m->nt);
  if (edge_nodes) memcpy(edge_nodes, m->en, sizeof(int32_t) * 2 * (size_t)m->ne);
  if (face_nodes) memcpy(face_nodes, m->fn, sizeof(int32_t) * 3 * (size_t)m->nf);
  if (tet_edges) memcpy(tet_edges, m->te, sizeof(int32_t) * 6 * (size_t)m->nt);
  if (tet_faces) memcpy(tet_faces, m->tf, sizeof(int32_t) * 4 * (size_t)m->nt);
  if (tet_nbr) memcpy(tet_nbr, m->nb, sizeof(int32_t) * 4 * (size_t)m->nt);
}

/* ---------------------------------------------------------------- locate */
static int inside(const omesh *m, int32_t t, const double *r) {
  double lam[4];
  or_bary(m, t, r, lam);
  return lam[0] >= 0.0 && lam[1] >= 0.0 && lam[2] >= 0.0 && lam[3] >= 0.0;
}

int32_t or_locate_brute_one(const void *h, const double *r) {
  const omesh *m = (const omesh *)h;
  for (int64_t t = 0; t < m->nt; t++)
    if (inside(m, (int32_t)t, r)) return (int32_t)t;
  return -1;
}

/* Smallest-id containing tet for each point; brute != 0 scans every tet. */
void or_locate(const void *h, int64_t n, const double *x, const double *y, const double *z,
               int32_t *tet, uint8_t *status, int32_t brute) {
  const omesh *m = (const omesh *)h;
  for (int64_t p = 0; p < n; p++) {
    double r[3] = {x[p], y[p], z[p]};
    int32_t found = -1;
    if (brute) {
      found = or_locate_brute_one(h, r);
    } else if (isfinite(r[0]) && isfinite(r[1]) && isfinite(r[2])) {
      int64_t c = cell_of(m, 0, r[0]) +
                  (int64_t)m->gd[0] * (cell_of(m, 1, r[1]) + (int64_t)m->gd[1] * cell_of(m, 2, r[2]));
      for (int64_t i = m->gstart[c]; i < m->gstart[c + 1]; i++)
        if (inside(m, m->gtet[i], r)) { found = m->gtet[i]; break; }
    }
    tet[p] = found;
    if (status) status[p] = found < 0 ? OR_LOST : OR_OK;
  }
}

/* --------------------------------------------------------------- Whitney */
void or_whitney1(const void *h, int32_t t, const double *r, double *W /*[6][3]*/) {
  const omesh *m = (const omesh *)h;
  double lam[4];
  or_bary(m, t, r, lam);
  const double *g = m->gl + 12 * (int64_t)t;
  for (int e = 0; e < 6; e++) {
    int i = LE[e][0], j = LE[e][1];
    for (int a = 0; a < 3; a++) W[3 * e + a] = lam[i] * g[3 * j + a] - lam[j] * g[3 * i + a];
  }
}

void or_whitney2(const void *h, int32_t t, const double *r, double *W /*[4][3]*/) {
  const omesh *m = (const omesh *)h;
  double lam[4];
  or_bary(m, t, r, lam);
  const double *g = m->gl + 12 * (int64_t)t;
  for (int f = 0; f < 4; f++) {
    int i = LF[f][0], j = LF[f][1], l = LF[f][2];
    double cjl[3], cli[3], cij[3];
    cross3(g + 3 * j, g + 3 * l, cjl);
    cross3(g + 3 * l, g + 3 * i, cli);
    cross3(g + 3 * i, g + 3 * j, cij);
    for (int a = 0; a < 3; a++)
      W[3 * f + a] = 2.0 * ((lam[i] * cjl[a] + lam[j] * cli[a]) + lam[l] * cij[a]);
  }
}

/* Envelope fields at r in tet t from complex128 DoFs (interleaved re,im).
 * Et, Bt: [re_x, re_y, re_z, im_x, im_y, im_z]. */
void or_gather(const void *h, int32_t t, const double *r, const double *e_dof, const double *b_dof,
               double *Et, double *Bt) {
  const omesh *m = (const omesh *)h;
  double W1[18], W2[12];
  or_whitney1(h, t, r, W1);
  or_whitney2(h, t, r, W2);
  for (int i = 0; i < 6; i++) { Et[i] = 0.0; Bt[i] = 0.0; }
  for (int e = 0; e < 6; e++) {
    int64_t id = m->te[6 * (int64_t)t + e];
    double re = e_dof[2 * id], im = e_dof[2 * id + 1];
    for (int a = 0; a < 3; a++) {
      Et[a] = Et[a] + re * W1[3 * e + a];
      Et[3 + a] = Et[3 + a] + im * W1[3 * e + a];
    }
  }
  for (int f = 0; f < 4; f++) {
    int64_t id = m->tf[4 * (int64_t)t + f];
    double re = b_dof[2 * id], im = b_dof[2 * id + 1];
    for (int a = 0; a < 3; a++) {
      Bt[a] = Bt[a] + re * W2[3 * f + a];
      Bt[3 + a] = Bt[3 + a] + im * W2[3 * f + a];
    }
  }
}

/* ---------------------------------------------------------------- deposit */
static void deposit_segment(const omesh *m, int32_t t, const double *la, const double *lb, double qw,
                            double *dG) {
  for (int e = 0; e < 6; e++) {
    int i = LE[e][0], j = LE[e][1];
    double t1 = la[i] * lb[j];
    double t2 = la[j] * lb[i];
    dG[m->te[6 * (int64_t)t + e]] += qw * (t1 - t2);
  }
}

/* ------------------------------------------------------------------ step */
typedef struct {
  double *x, *y, *z, *vx, *vy, *vz;
  int32_t *tet;
  uint8_t *status;
  int32_t *n_cross;
} oparts;

static int finite3(const double *a) { return isfinite(a[0]) && isfinite(a[1]) && isfinite(a[2]); }

static void step_one(const omesh *m, oparts *P, int64_t p, double kq, double qw, double cre, double cim,
                     const double *e_dof, const double *b_dof, double dt, int32_t max_cross,
                     int32_t wall_mode, double *dG, uint8_t *mirror) {
  int32_t T = P->tet[p];
  if (T < 0) return;
  if (T >= m->nt) { P->tet[p] = -1; P->status[p] = OR_LOST; return; }
  double a[3] = {P->x[p], P->y[p], P->z[p]};
  double v[3] = {P->vx[p], P->vy[p], P->vz[p]};
  /* (b) gather + (c) carrier */
  double Et[6], Bt[6], E[3], B[3];
  or_gather(m, T, a, e_dof, b_dof, Et, Bt);
  for (int c = 0; c < 3; c++) {
    E[c] = cre * Et[c] - cim * Et[3 + c];
    B[c] = cre * Bt[c] - cim * Bt[3 + c];
  }
  /* (d) Boris */
  double vm[3], tau[3], s[3], vp[3], vpl[3], vn[3], b[3], cr[3];
  for (int c = 0; c < 3; c++) vm[c] = v[c] + kq * E[c];
  for (int c = 0; c < 3; c++) tau[c] = kq * B[c];
  double t2 = (tau[0] * tau[0] + tau[1] * tau[1]) + tau[2] * tau[2];
  double f = 2.0 / (1.0 + t2);
  for (int c = 0; c < 3; c++) s[c] = f * tau[c];
  cross3(vm, tau, cr);
  for (int c = 0; c < 3; c++) vp[c] = vm[c] + cr[c];
  cross3(vp, s, cr);
  for (int c = 0; c < 3; c++) vpl[c] = vm[c] + cr[c];
  for (int c = 0; c < 3; c++) vn[c] = vpl[c] + kq * E[c];
  for (int c = 0; c < 3; c++) b[c] = a[c] + dt * vn[c];
  if (!finite3(vn) || !finite3(b)) { P->status[p] = OR_NONFINITE; P->tet[p] = -2 - T; return; }
  /* (e) track + (f) deposit */
  double la[4], lb[4], lp[4];
  or_bary(m, T, a, la);
  int entry = -1;
  int32_t ncross = 0;
  int mir = 0;   /* bit ax: mirrored in axis ax an odd number of times */
  for (;;) {
    or_bary(m, T, b, lb);
    int kx = -1;
    double smin = INFINITY;
    for (int k = 0; k < 4; k++) {
      if (k == entry || !(lb[k] < 0.0)) continue;
      double sk = la[k] / (la[k] - lb[k]);
      if (sk < 0.0) sk = 0.0;
      if (sk < smin) { smin = sk; kx = k; }
    }
    if (kx < 0) {
      deposit_segment(m, T, la, lb, qw, dG);
      a[0] = b[0]; a[1] = b[1]; a[2] = b[2];
      break;
    }
    double pp[3];
    for (int c = 0; c < 3; c++) pp[c] = a[c] + smin * (b[c] - a[c]);
    for (int i = 0; i < 4; i++) lp[i] = (i == kx) ? 0.0 : la[i] + smin * (lb[i] - la[i]);
    deposit_segment(m, T, la, lp, qw, dG);
    ncross++;
    a[0] = pp[0]; a[1] = pp[1]; a[2] = pp[2];
    if (ncross > max_cross) { P->status[p] = OR_CAP; T = -2 - T; break; }
    int32_t nbt = m->nb[4 * (int64_t)T + kx];
    if (nbt >= 0) {
      const int32_t *on = m->tn + 4 * (int64_t)T;
      const int32_t *nn = m->tn + 4 * (int64_t)nbt;
      int ent = -1;
      for (int i2 = 0; i2 < 4; i2++) {
        int hit = -1;
        for (int i = 0; i < 4; i++)
          if (on[i] == nn[i2]) hit = i;
        if (hit >= 0) la[i2] = lp[hit];
        else { la[i2] = 0.0; ent = i2; }
      }
      T = nbt;
      entry = ent;
    } else if (nbt <= -1 && nbt >= -6 && wall_mode == 0) {
      int code = -1 - nbt, ax = code / 2, side = code % 2;
      double L = side ? m->hi[ax] : m->lo[ax];
      b[ax] = 2.0 * L - b[ax];
      vn[ax] = -vn[ax];
      mir ^= 1 << ax;
      for (int i = 0; i < 4; i++) la[i] = lp[i];
      entry = kx;
    } else {
      P->status[p] = OR_ABSORBED;
      T = -2 - T;
      break;
    }
  }
  P->x[p] = a[0]; P->y[p] = a[1]; P->z[p] = a[2];
  P->vx[p] = vn[0]; P->vy[p] = vn[1]; P->vz[p] = vn[2];
  P->tet[p] = T;
  if (P->n_cross) P->n_cross[p] += ncross;
  if (mirror) mirror[p] = (uint8_t)mir;
}

/* One particle step for all particles, serially in index order.
 * Species s covers particles [species_begin[s], species_begin[s+1]).
 * dG (length ne) is accumulated into (not cleared).  mirror (length n, may be
 * NULL) receives per particle the axes whose velocity component the walls
 * mirrored an odd number of times during the step (bit ax), recorded where
 * the walk reflects; particles not stepped keep their entry. */
int or_push_step(const void *h, int64_t n, double *x, double *y, double *z, double *vx, double *vy,
                 double *vz, int32_t *tet, uint8_t *status, int32_t *n_cross, int32_t n_species,
                 const int64_t *species_begin, const double *q, const double *mass, const double *w,
                 const double *e_dof, const double *b_dof, double amp, double omega0, double t,
                 double dt, int32_t max_cross, int32_t wall_mode, double *dG, uint8_t *mirror) {
  const omesh *m = (const omesh *)h;
  oparts P = {x, y, z, vx, vy, vz, tet, status, n_cross};
  double phi = omega0 * t;
  double cre = amp * cos(phi), cim = amp * sin(phi);
  for (int32_t s = 0; s < n_species; s++) {
    double kq = ((q[s] / mass[s]) * dt) * 0.5;
    double qw = q[s] * w[s];
    int64_t p1 = species_begin[s + 1] < n ? species_begin[s + 1] : n;
    for (int64_t p = species_begin[s]; p < p1; p++)
      step_one(m, &P, p, kq, qw, cre, cim, e_dof, b_dof, dt, max_cross, wall_mode, dG, mirror);
  }
  return 0;
}

/* ----------------------------------------------------------- diagnostics */
/* Whitney-0 nodal charge rho_n = sum_p q w lambda_n(r_p) over particles with
 * a known tet (active, or frozen with tet = -2 - T). */
void or_nodal_charge(const void *h, int64_t n, const double *x, const double *y, const double *z,
                     const int32_t *tet, int32_t n_species, const int64_t *species_begin,
                     const double *q, const double *w, double *rho) {
  const omesh *m = (const omesh *)h;
  memset(rho, 0, sizeof(double) * (size_t)m->nn);
  for (int32_t s = 0; s < n_species; s++) {
    double qw = q[s] * w[s];
    int64_t p1 = species_begin[s + 1] < n ? species_begin[s + 1] : n;
    for (int64_t p = species_begin[s]; p < p1; p++) {
      int32_t T = tet[p];
      if (T == -1) continue;
      if (T < 0) T = -2 - T;
      if (T >= m->nt) continue;
      double r[3] = {x[p], y[p], z[p]}, lam[4];
      or_bary(m, T, r, lam);
      for (int i = 0; i < 4; i++) rho[m->tn[4 * (int64_t)T + i]] += qw * lam[i];
    }
  }
}

/* Discrete divergence with the edge-to-node incidence D (edge i->j: +1 at j,
 * -1 at i): out = D^T G. */
void or_edge_divergence(const void *h, const double *G, double *out) {
  const omesh *m = (const omesh *)h;
  memset(out, 0, sizeof(double) * (size_t)m->nn);
  for (int64_t e = 0; e < m->ne; e++) {
    out[m->en[2 * e + 1]] += G[e];
    out[m->en[2 * e]] -= G[e];
  }
}

/* Face circulation of edge values: out_f = v_ij + v_jk - v_ik (curl incidence C). */
void or_face_circulation(const void *h, const double *v, double *out) {
  const omesh *m = (const omesh *)h;
  int64_t *keys = malloc(sizeof(int64_t) * (size_t)m->ne);
  for (int64_t e = 0; e < m->ne; e++) keys[e] = (int64_t)m->en[2 * e] * m->nn + m->en[2 * e + 1];
  for (int64_t f = 0; f < m->nf; f++) {
    int64_t i = m->fn[3 * f], j = m->fn[3 * f + 1], k = m->fn[3 * f + 2];
    int64_t eij = find_i64(keys, m->ne, i * m->nn + j);
    int64_t ejk = find_i64(keys, m->ne, j * m->nn + k);
    int64_t eik = find_i64(keys, m->ne, i * m->nn + k);
    out[f] = (v[eij] + v[ejk]) - v[eik];
  }
  free(keys);
}

/* Envelope-frame map of the time-integrated current: out = e^{-j omega0 t} G
 * (interleaved complex128). */
void or_envelope_frame(int64_t ne, const double *G, double omega0, double t, double *out) {
  double phi = omega0 * t, c = cos(phi), s = sin(phi);
  for (int64_t e = 0; e < ne; e++) {
    out[2 * e] = c * G[e];
    out[2 * e + 1] = -(s * G[e]);
  }
}

double or_kinetic_energy(int64_t n, const double *vx, const double *vy, const double *vz,
                         const int32_t *tet, int32_t n_species, const int64_t *species_begin,
                         const double *mass, const double *w) {
  double ke = 0.0;
  for (int32_t s = 0; s < n_species; s++) {
    int64_t p1 = species_begin[s + 1] < n ? species_begin[s + 1] : n;
    for (int64_t p = species_begin[s]; p < p1; p++) {
      if (tet && tet[p] < 0) continue;
      double v2 = (vx[p] * vx[p] + vy[p] * vy[p]) + vz[p] * vz[p];
      ke += (0.5 * mass[s] * w[s]) * v2;
    }
  }
  return ke;
}

/* ------------------------------------------------------------------ JVP */
/* Forward-mode tangent of one step, for checking gradients.  The values
 * follow exactly the path of or_push_step (same tets, crossings and wall
 * events); the tangents (dr, dv) and the tangent DoFs (de, db, complex
 * interleaved like the DoFs) are propagated through every smooth operation:
 *   dE~ = sum_e de_e W1_e(r) + sum_e e_e (dW1_e/dr) dr,
 *     with (dW1_ij/dr) dr = (gl_i . dr) gl_j - (gl_j . dr) gl_i;
 *   dB~ = sum_f db_f W2_f(r) + sum_f b_f (dW2_f/dr) dr,
 *     with (dW2_ijl/dr) dr = 2 ((gl_i . dr) c_jl + (gl_j . dr) c_li + (gl_l . dr) c_ij);
 *   the carrier product, every Boris operation, r + dt v, and at a wall the
 *   mirrored component.  A particle frozen at a crossing point gets the
 *   tangent of that point (through the tangent of the exit parameter).
 * The tet sequence is held fixed: this is the derivative of the piecewise
 * smooth map on the piece the values lie in. */
static void tangent_fields(const omesh *m, int32_t T, const double *r, const double *dr, const double *e_dof,
                           const double *b_dof, const double *de, const double *dbf, double *dEt, double *dBt) {
  double W1[18], W2[12], lam[4];
  or_whitney1(m, T, r, W1);
  or_whitney2(m, T, r, W2);
  or_bary(m, T, r, lam);
  const double *g = m->gl + 12 * (int64_t)T;
  double gd[4];
  for (int k = 0; k < 4; k++) gd[k] = (g[3 * k] * dr[0] + g[3 * k + 1] * dr[1]) + g[3 * k + 2] * dr[2];
  for (int i = 0; i < 6; i++) { dEt[i] = 0.0; dBt[i] = 0.0; }
  for (int e = 0; e < 6; e++) {
    int64_t id = m->te[6 * (int64_t)T + e];
    int i = LE[e][0], j = LE[e][1];
    for (int a = 0; a < 3; a++) {
      double dW = gd[i] * g[3 * j + a] - gd[j] * g[3 * i + a];
      dEt[a] += de[2 * id] * W1[3 * e + a] + e_dof[2 * id] * dW;
      dEt[3 + a] += de[2 * id + 1] * W1[3 * e + a] + e_dof[2 * id + 1] * dW;
    }
  }
  for (int f = 0; f < 4; f++) {
    int64_t id = m->tf[4 * (int64_t)T + f];
    int i = LF[f][0], j = LF[f][1], l = LF[f][2];
    double cjl[3], cli[3], cij[3];
    cross3(g + 3 * j, g + 3 * l, cjl);
    cross3(g + 3 * l, g + 3 * i, cli);
    cross3(g + 3 * i, g + 3 * j, cij);
    for (int a = 0; a < 3; a++) {
      double dW = 2.0 * ((gd[i] * cjl[a] + gd[j] * cli[a]) + gd[l] * cij[a]);
      dBt[a] += dbf[2 * id] * W2[3 * f + a] + b_dof[2 * id] * dW;
      dBt[3 + a] += dbf[2 * id + 1] * W2[3 * f + a] + b_dof[2 * id + 1] * dW;
    }
  }
}

static double dot3(const double *a, const double *b) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }

/* Tangent of one piece's deposit: with lambda_i = lambda_i(start), mu_i =
 * lambda_i(end) and their tangents dl_i = gl_i . d(start), dm_i = gl_i .
 * d(end) in this tet, d g_ij = q w (dl_i mu_j + lambda_i dm_j - dl_j mu_i -
 * lambda_j dm_i). */
static void deposit_segment_tangent(const omesh *m, int32_t t, const double *la, const double *lb,
                                    const double *dpa, const double *dpb, double qw, double *dGt) {
  if (!dGt) return;
  const double *g = m->gl + 12 * (int64_t)t;
  double dl[4], dm[4];
  for (int k = 0; k < 4; k++) {
    dl[k] = (g[3 * k] * dpa[0] + g[3 * k + 1] * dpa[1]) + g[3 * k + 2] * dpa[2];
    dm[k] = (g[3 * k] * dpb[0] + g[3 * k + 1] * dpb[1]) + g[3 * k + 2] * dpb[2];
  }
  for (int e = 0; e < 6; e++) {
    int i = LE[e][0], j = LE[e][1];
    double v = ((dl[i] * lb[j] + la[i] * dm[j]) - dl[j] * lb[i]) - la[j] * dm[i];
    dGt[m->te[6 * (int64_t)t + e]] += qw * v;
  }
}

static void step_one_jvp(const omesh *m, oparts *P, int64_t p, double kq, double qw, double cre, double cim,
                         const double *e_dof, const double *b_dof, double dt, int32_t max_cross, int32_t wall_mode,
                         double *dG, double *TR, double *TV, const double *de, const double *dbf, double *dGt) {
  int32_t T = P->tet[p];
  if (T < 0) return;
  if (T >= m->nt) { P->tet[p] = -1; P->status[p] = OR_LOST; return; }
  double a[3] = {P->x[p], P->y[p], P->z[p]};
  double v[3] = {P->vx[p], P->vy[p], P->vz[p]};
  double da[3] = {TR[3 * p], TR[3 * p + 1], TR[3 * p + 2]};
  double dv[3] = {TV[3 * p], TV[3 * p + 1], TV[3 * p + 2]};
  double Et[6], Bt[6], E[3], B[3], dEt[6], dBt[6], dE[3], dB[3];
  or_gather(m, T, a, e_dof, b_dof, Et, Bt);
  tangent_fields(m, T, a, da, e_dof, b_dof, de, dbf, dEt, dBt);
  for (int c = 0; c < 3; c++) {
    E[c] = cre * Et[c] - cim * Et[3 + c];
    B[c] = cre * Bt[c] - cim * Bt[3 + c];
    dE[c] = cre * dEt[c] - cim * dEt[3 + c];
    dB[c] = cre * dBt[c] - cim * dBt[3 + c];
  }
  double vm[3], tau[3], s[3], vp[3], vpl[3], vn[3], b[3], cr[3];
  double dvm[3], dtau[3], ds[3], dvp[3], dvpl[3], dvn[3], db[3], c1[3], c2[3];
  for (int c = 0; c < 3; c++) { vm[c] = v[c] + kq * E[c]; dvm[c] = dv[c] + kq * dE[c]; }
  for (int c = 0; c < 3; c++) { tau[c] = kq * B[c]; dtau[c] = kq * dB[c]; }
  double t2 = (tau[0] * tau[0] + tau[1] * tau[1]) + tau[2] * tau[2];
  double dt2 = 2.0 * dot3(tau, dtau);
  double f = 2.0 / (1.0 + t2);
  double df = -0.5 * f * f * dt2;
  for (int c = 0; c < 3; c++) { s[c] = f * tau[c]; ds[c] = df * tau[c] + f * dtau[c]; }
  cross3(vm, tau, cr);
  cross3(dvm, tau, c1);
  cross3(vm, dtau, c2);
  for (int c = 0; c < 3; c++) { vp[c] = vm[c] + cr[c]; dvp[c] = dvm[c] + c1[c] + c2[c]; }
  cross3(vp, s, cr);
  cross3(dvp, s, c1);
  cross3(vp, ds, c2);
  for (int c = 0; c < 3; c++) { vpl[c] = vm[c] + cr[c]; dvpl[c] = dvm[c] + c1[c] + c2[c]; }
  for (int c = 0; c < 3; c++) { vn[c] = vpl[c] + kq * E[c]; dvn[c] = dvpl[c] + kq * dE[c]; }
  for (int c = 0; c < 3; c++) { b[c] = a[c] + dt * vn[c]; db[c] = da[c] + dt * dvn[c]; }
  if (!finite3(vn) || !finite3(b)) { P->status[p] = OR_NONFINITE; P->tet[p] = -2 - T; return; }
  double la[4], lb[4], lp[4];
  or_bary(m, T, a, la);
  int entry = -1;
  int32_t ncross = 0;
  for (;;) {
    or_bary(m, T, b, lb);
    int kx = -1;
    double smin = INFINITY;
    for (int k = 0; k < 4; k++) {
      if (k == entry || !(lb[k] < 0.0)) continue;
      double sk = la[k] / (la[k] - lb[k]);
      if (sk < 0.0) sk = 0.0;
      if (sk < smin) { smin = sk; kx = k; }
    }
    if (kx < 0) {
      deposit_segment(m, T, la, lb, qw, dG);
      deposit_segment_tangent(m, T, la, lb, da, db, qw, dGt);
      for (int c = 0; c < 3; c++) { a[c] = b[c]; da[c] = db[c]; }
      break;
    }
    /* tangent of the exit parameter s = la_k / (la_k - lb_k), with the
     * barycentric tangents of the piece ends taken from their positions */
    const double *g = m->gl + 12 * (int64_t)T;
    double dla = (g[3 * kx] * da[0] + g[3 * kx + 1] * da[1]) + g[3 * kx + 2] * da[2];
    double dlb = (g[3 * kx] * db[0] + g[3 * kx + 1] * db[1]) + g[3 * kx + 2] * db[2];
    double den = la[kx] - lb[kx];
    double dsm = (smin > 0.0) ? (dla * den - la[kx] * (dla - dlb)) / (den * den) : 0.0;
    double pp[3], dpp[3];
    for (int c = 0; c < 3; c++) {
      pp[c] = a[c] + smin * (b[c] - a[c]);
      dpp[c] = da[c] + dsm * (b[c] - a[c]) + smin * (db[c] - da[c]);
    }
    for (int i = 0; i < 4; i++) lp[i] = (i == kx) ? 0.0 : la[i] + smin * (lb[i] - la[i]);
    deposit_segment(m, T, la, lp, qw, dG);
    deposit_segment_tangent(m, T, la, lp, da, dpp, qw, dGt);
    ncross++;
    for (int c = 0; c < 3; c++) { a[c] = pp[c]; da[c] = dpp[c]; }
    if (ncross > max_cross) { P->status[p] = OR_CAP; T = -2 - T; break; }
    int32_t nbt = m->nb[4 * (int64_t)T + kx];
    if (nbt >= 0) {
      const int32_t *on = m->tn + 4 * (int64_t)T;
      const int32_t *nn = m->tn + 4 * (int64_t)nbt;
      int ent = -1;
      for (int i2 = 0; i2 < 4; i2++) {
        int hit = -1;
        for (int i = 0; i < 4; i++)
          if (on[i] == nn[i2]) hit = i;
        if (hit >= 0) la[i2] = lp[hit];
        else { la[i2] = 0.0; ent = i2; }
      }
      T = nbt;
      entry = ent;
    } else if (nbt <= -1 && nbt >= -6 && wall_mode == 0) {
      int code = -1 - nbt, ax = code / 2, side = code % 2;
      double L = side ? m->hi[ax] : m->lo[ax];
      b[ax] = 2.0 * L - b[ax];
      db[ax] = -db[ax];
      vn[ax] = -vn[ax];
      dvn[ax] = -dvn[ax];
      for (int i = 0; i < 4; i++) la[i] = lp[i];
      entry = kx;
    } else {
      P->status[p] = OR_ABSORBED;
      T = -2 - T;
      break;
    }
  }
  P->x[p] = a[0]; P->y[p] = a[1]; P->z[p] = a[2];
  P->vx[p] = vn[0]; P->vy[p] = vn[1]; P->vz[p] = vn[2];
  P->tet[p] = T;
  if (P->n_cross) P->n_cross[p] += ncross;
  for (int c = 0; c < 3; c++) { TR[3 * p + c] = da[c]; TV[3 * p + c] = dv[c] = dvn[c]; }
}

/* One step of values and tangents.  tr, tv: [n][3] tangents of position and
 * velocity, updated in place; de, db: tangent DoFs (complex interleaved);
 * dGt (length ne, may be NULL): the tangent of the step's deposit is added
 * to it. */
int or_push_step_jvp(const void *h, int64_t n, double *x, double *y, double *z, double *vx, double *vy,
                     double *vz, int32_t *tet, uint8_t *status, int32_t *n_cross, int32_t n_species,
                     const int64_t *species_begin, const double *q, const double *mass, const double *w,
                     const double *e_dof, const double *b_dof, double amp, double omega0, double t,
                     double dt, int32_t max_cross, int32_t wall_mode, double *dG, double *tr, double *tv,
                     const double *de, const double *db, double *dGt) {
  const omesh *m = (const omesh *)h;
  oparts P = {x, y, z, vx, vy, vz, tet, status, n_cross};
  double phi = omega0 * t;
  double cre = amp * cos(phi), cim = amp * sin(phi);
  for (int32_t s = 0; s < n_species; s++) {
    double kq = ((q[s] / mass[s]) * dt) * 0.5;
    double qw = q[s] * w[s];
    int64_t p1 = species_begin[s + 1] < n ? species_begin[s + 1] : n;
    for (int64_t p = species_begin[s]; p < p1; p++)
      step_one_jvp(m, &P, p, kq, qw, cre, cim, e_dof, b_dof, dt, max_cross, wall_mode, dG, tr, tv, de, db, dGt);
  }
  return 0;
}
