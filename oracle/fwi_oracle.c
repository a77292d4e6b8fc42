/*
 * fwi_oracle.c -- plain FP64 CPU oracle for the per-shot material gradient of
 * Fathi, Kallivokas & Poursartip, "Full-waveform inversion in
 * three-dimensional PML-truncated elastic media" (arXiv:1504.08340).
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and the CPU legs
 * of bench.py (cpu_baseline, --impl reference) may load this library. The
 * product (the CUDA library) never links, loads or calls it, and the two share
 * no code, header, table or helper.
 *
 * What it computes, in the paper's order:
 *   Sec. 2, Eqs. (3a)/(3b): Galerkin weak form, discretised with 27-node
 *     hexahedral spectral elements and Legendre-Gauss-Lobatto (LGL) quadrature
 *     (quadrature points = nodes), so the mass-like matrices are diagonal.
 *     Every operator below is an element loop over the quadrature points,
 *     written as the quadrature of the weak-form integrand.
 *   Eq. (5)/(6): semi-discrete system M d'' + C d' + K d + G dbar = f with
 *     d = (u, S), integrated as the first-order system (6) by classic RK4.
 *   Eq. (7): misfit J, receivers at nodes.
 *   Eq. (14)/(15) and Appendix B: the adjoint problem with the TRANSPOSED
 *     system matrices, integrated backwards in time by the reverse RK4 stages
 *     of Appendix B.
 *   Eq. (18), Appendix C (C.1a, C.1f, C.1g): misfit part of the lambda / mu
 *     gradients, restricted to the regular (interior) domain, and the lumped
 *     mass-like matrix Mtilde.
 *   Eqs. (8), (9) with (C.1b)-(C.1e): Tikhonov and total-variation
 *     regularisation terms and their gradients on the interior nodal field.
 *
 * Readings where the paper is silent, defers to its companion paper [13], or is
 * garbled (each is also listed in the design notes):
 *   R1 PML coefficients (Sec. 2 only says "products of certain elements of the
 *      stretch tensors"): with stretch functions eps_s = alpha_s + beta_s/(i w),
 *      alpha_s = 1 + alpha0 (l_s/L)^m, beta_s = beta0 (l_s/L)^m,
 *        a + b/(iw) + c/(iw)^2 + d/(iw)^3 = eps_x eps_y eps_z,
 *        Lambda_e + Lambda_p/(iw) + Lambda_w/(iw)^2
 *              = diag(eps_y eps_z, eps_x eps_z, eps_x eps_y).
 *   R2 S is continuous and nodal with 6 symmetric components on every node of
 *      a PML element (matches the state counts printed in Sec. 4.2 and 4.5).
 *   R3 Appendix B drops the transposes of (15); they are put back: the reverse
 *      RK4 applies G^T, K^T, C^T. y0 is the history measured from T
 *      (y0(T) = 0, d y0/dt = y1), which is what (15) and its final values say.
 *   R4 the forcing at half steps (f^{n-1/2} in Appendix B) is the average of
 *      the two neighbouring step values (linear interpolation).
 *   R5 the time integrals in J and in (C.1f)/(C.1g) use the trapezoid rule on
 *      the step grid.
 *   R6 PML material is the value at the nearest interface node (index clamp),
 *      and the gradient is restricted to interior elements (Sec. 3.1.3).
 *   R7 (13b) writes "c S" where the adjoint stress T is meant; T is used.
 *   R8 (17a)/(17b) and (C.1d)/(C.1e) are the derivative of
 *      R int (|grad f|^2 + eps)^(1/2), i.e. of (9) without its factor 1/2; the TV
 *      functional is taken as that, so that the gradient is its derivative. The
 *      denominator of (C.1d)/(C.1e) is read pointwise: |grad f_h|^2 at the
 *      quadrature point. TN (8) and (16), (C.1b)/(C.1c) agree as printed.
 *
 * Pins: see tests/test_oracle_*.py (stiffness symmetry and rigid modes, patch
 * test, transposes by the dot-product test, RK4 against the exact amplification
 * of an eigenmode, energy, state counts printed in Sec. 4.2 / 4.5, directional
 * finite differences as in Sec. 4.1 / Table 2; the PML coupling operators and
 * lumped a, b, c, d against the stretched-coordinate stress and divergence in the
 * Laplace domain, the identity-stretch patch test across the interface, the
 * wavelet's closed forms, trivial forward cases, PML reflection against a wider
 * domain, and Stokes' point-force solution in a homogeneous full space).
 * Parity unpinned: the absolute values of Table 2 (trial model, PML details
 * of [13] and the data mesh are not given in the paper).
 *
 * State layout (oracle's own): Y[level][node][9], level 0 = history (x0),
 * 1 = value (x1), 2 = rate (x2); per node u_x,u_y,u_z, S_xx,S_yy,S_zz,S_yz,
 * S_xz,S_xy. Nodes are numbered (k * ny_nodes + j) * nx_nodes + i, i along x,
 * k along depth (k = 0 is the ground surface).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NV 9 /* per node: 3 displacement + 6 stress components */

/* one-dimensional LGL rule on [-1,1] with nodes -1, 0, 1 */
static const double GLL_W[3] = {1.0 / 3.0, 4.0 / 3.0, 1.0 / 3.0};
/* D1[q][a] = derivative of the quadratic Lagrange polynomial of node a at node q */
static const double D1[3][3] = {{-1.5, 2.0, -0.5}, {-0.5, 0.0, 0.5}, {0.5, -2.0, 1.5}};

/* symmetric tensor component index of (i,j): xx yy zz yz xz xy */
static const int SYM[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};

typedef struct orc_mesh {
  int nel[3]; /* interior elements per axis */
  int npml, top_pml;
  double h, rho, alpha0, beta0;
  int pml_m;
  int N[3];  /* elements per axis */
  int nn[3]; /* nodes per axis */
  int lo[3], hi[3]; /* interior element range [lo,hi) per axis */
  long nnode;
  long nmat; /* interior (material) nodes */
  double *lam, *mu; /* nodal, every node (extended into the PML) */
  double *al[3], *be[3]; /* stretch functions at node coordinates, per axis */
  unsigned char *pml_node, *dir_node;
  double *Mu, *Cu, *Ku, *Gu; /* lumped u-row diagonals */
  double *Ms, *Cs, *Ks, *Gs; /* lumped S-row diagonals */
  double *Mtilde; /* (C.1a) on material nodes */
  int nthreads;
} orc_mesh;

/* ------------------------------------------------------------------ mesh */

static long node_id(const orc_mesh *m, int i, int j, int k) {
  return ((long)k * m->nn[1] + j) * m->nn[0] + i;
}

static int elem_is_rd(const orc_mesh *m, int ex, int ey, int ez) {
  return ex >= m->lo[0] && ex < m->hi[0] && ey >= m->lo[1] && ey < m->hi[1] &&
         ez >= m->lo[2] && ez < m->hi[2];
}

/* distance into the PML of node coordinate c (in half-element units) along axis ax */
static double pml_depth(const orc_mesh *m, int ax, int c) {
  int a = 2 * m->lo[ax], b = 2 * m->hi[ax];
  if (c < a) return (a - c) * 0.5 * m->h;
  if (c > b) return (c - b) * 0.5 * m->h;
  return 0.0;
}

static void coef_at(const orc_mesh *m, long g, double *a, double *b, double *c,
                    double *d, double Le[3], double Lp[3], double Lw[3]) {
  int i = (int)(g % m->nn[0]);
  int j = (int)((g / m->nn[0]) % m->nn[1]);
  int k = (int)(g / ((long)m->nn[0] * m->nn[1]));
  double ax = m->al[0][i], ay = m->al[1][j], az = m->al[2][k];
  double bx = m->be[0][i], by = m->be[1][j], bz = m->be[2][k];
  if (a) *a = ax * ay * az;
  if (b) *b = ax * ay * bz + ax * by * az + bx * ay * az;
  if (c) *c = ax * by * bz + bx * ay * bz + bx * by * az;
  if (d) *d = bx * by * bz;
  if (Le) { Le[0] = ay * az; Le[1] = ax * az; Le[2] = ax * ay; }
  if (Lp) { Lp[0] = ay * bz + by * az; Lp[1] = ax * bz + bx * az; Lp[2] = ax * by + bx * ay; }
  if (Lw) { Lw[0] = by * bz; Lw[1] = bx * bz; Lw[2] = bx * by; }
}

/* global node of local node (a0,a1,a2) of element (ex,ey,ez) */
static long elem_node(const orc_mesh *m, int ex, int ey, int ez, int a0, int a1, int a2) {
  return node_id(m, 2 * ex + a0, 2 * ey + a1, 2 * ez + a2);
}

/* d phi_a / d x_j at quadrature point q (both local multi-indices); zero off the line */
static double dphi(const orc_mesh *m, const int a[3], const int q[3], int j) {
  for (int k = 0; k < 3; k++)
    if (k != j && a[k] != q[k]) return 0.0;
  return (2.0 / m->h) * D1[q[j]][a[j]];
}

static double quad_weight(const orc_mesh *m, const int q[3]) {
  double hj = 0.5 * m->h;
  return GLL_W[q[0]] * GLL_W[q[1]] * GLL_W[q[2]] * hj * hj * hj;
}

orc_mesh *orc_create(int nx, int ny, int nz, int npml, int top_pml, double h,
                     double rho, double alpha0, double beta0, int pml_m) {
  if (nx < 1 || ny < 1 || nz < 1 || npml < 0 || h <= 0 || rho <= 0) return NULL;
  orc_mesh *m = (orc_mesh *)calloc(1, sizeof(orc_mesh));
  m->nel[0] = nx; m->nel[1] = ny; m->nel[2] = nz;
  m->npml = npml; m->top_pml = top_pml ? 1 : 0;
  m->h = h; m->rho = rho; m->alpha0 = alpha0; m->beta0 = beta0; m->pml_m = pml_m;
  m->N[0] = nx + 2 * npml; m->N[1] = ny + 2 * npml;
  m->N[2] = nz + npml + (m->top_pml ? npml : 0);
  m->lo[0] = npml; m->lo[1] = npml; m->lo[2] = m->top_pml ? npml : 0;
  for (int a = 0; a < 3; a++) {
    m->hi[a] = m->lo[a] + m->nel[a];
    m->nn[a] = 2 * m->N[a] + 1;
  }
  m->nnode = (long)m->nn[0] * m->nn[1] * m->nn[2];
  m->nmat = (long)(2 * nx + 1) * (2 * ny + 1) * (2 * nz + 1);
  m->nthreads = 1;
  double L = npml * h;
  for (int a = 0; a < 3; a++) {
    m->al[a] = (double *)malloc(sizeof(double) * m->nn[a]);
    m->be[a] = (double *)malloc(sizeof(double) * m->nn[a]);
    for (int c = 0; c < m->nn[a]; c++) {
      double l = pml_depth(m, a, c);
      double r = (L > 0) ? pow(l / L, (double)pml_m) : 0.0;
      if (l == 0.0) r = 0.0;
      m->al[a][c] = 1.0 + alpha0 * r;
      m->be[a][c] = beta0 * r;
    }
  }
  m->pml_node = (unsigned char *)calloc(m->nnode, 1);
  m->dir_node = (unsigned char *)calloc(m->nnode, 1);
  for (int ez = 0; ez < m->N[2]; ez++)
    for (int ey = 0; ey < m->N[1]; ey++)
      for (int ex = 0; ex < m->N[0]; ex++) {
        if (elem_is_rd(m, ex, ey, ez)) continue;
        for (int c = 0; c < 27; c++)
          m->pml_node[elem_node(m, ex, ey, ez, c % 3, (c / 3) % 3, c / 9)] = 1;
      }
  for (int k = 0; k < m->nn[2]; k++)
    for (int j = 0; j < m->nn[1]; j++)
      for (int i = 0; i < m->nn[0]; i++) {
        int d = (i == 0 || i == m->nn[0] - 1 || j == 0 || j == m->nn[1] - 1 ||
                 k == m->nn[2] - 1 || (m->top_pml && k == 0));
        m->dir_node[node_id(m, i, j, k)] = (unsigned char)d;
      }
  m->lam = (double *)calloc(m->nnode, sizeof(double));
  m->mu = (double *)calloc(m->nnode, sizeof(double));
  double **diag[8] = {&m->Mu, &m->Cu, &m->Ku, &m->Gu, &m->Ms, &m->Cs, &m->Ks, &m->Gs};
  for (int t = 0; t < 8; t++) *diag[t] = (double *)calloc(m->nnode, sizeof(double));
  m->Mtilde = (double *)calloc(m->nmat, sizeof(double));
  /* lumped diagonals: the LGL quadrature of int coef * phi_a * phi_b, which is
   * diagonal because quadrature points coincide with nodes */
  for (int ez = 0; ez < m->N[2]; ez++)
    for (int ey = 0; ey < m->N[1]; ey++)
      for (int ex = 0; ex < m->N[0]; ex++) {
        int rd = elem_is_rd(m, ex, ey, ez);
        for (int c = 0; c < 27; c++) {
          int q[3] = {c % 3, (c / 3) % 3, c / 9};
          long g = elem_node(m, ex, ey, ez, q[0], q[1], q[2]);
          double wq = quad_weight(m, q);
          if (rd) {
            m->Mu[g] += wq * rho;
            int mi = 2 * (ex - m->lo[0]) + q[0], mj = 2 * (ey - m->lo[1]) + q[1],
                mk = 2 * (ez - m->lo[2]) + q[2];
            m->Mtilde[((long)mk * (2 * ny + 1) + mj) * (2 * nx + 1) + mi] += wq;
          } else {
            double a, b, cc, d;
            coef_at(m, g, &a, &b, &cc, &d, NULL, NULL, NULL);
            m->Mu[g] += wq * rho * a; m->Cu[g] += wq * rho * b;
            m->Ku[g] += wq * rho * cc; m->Gu[g] += wq * rho * d;
            m->Ms[g] += wq * a; m->Cs[g] += wq * b;
            m->Ks[g] += wq * cc; m->Gs[g] += wq * d;
          }
        }
      }
  return m;
}

void orc_destroy(orc_mesh *m) {
  if (!m) return;
  for (int a = 0; a < 3; a++) { free(m->al[a]); free(m->be[a]); }
  free(m->pml_node); free(m->dir_node); free(m->lam); free(m->mu);
  free(m->Mu); free(m->Cu); free(m->Ku); free(m->Gu);
  free(m->Ms); free(m->Cs); free(m->Ks); free(m->Gs); free(m->Mtilde);
  free(m);
}

void orc_set_threads(orc_mesh *m, int n) { m->nthreads = n > 0 ? n : 1; }

void orc_dims(const orc_mesh *m, long *out) {
  /* nodes per axis (3), elements per axis (3), nnode, nmat, lo(3), hi(3) */
  for (int a = 0; a < 3; a++) { out[a] = m->nn[a]; out[3 + a] = m->N[a]; }
  out[6] = m->nnode; out[7] = m->nmat;
  for (int a = 0; a < 3; a++) { out[8 + a] = m->lo[a]; out[11 + a] = m->hi[a]; }
}

/* material on interior nodes [k][j][i] -> every node, extended into the PML by
 * the value at the nearest interface node (reading R6) */
int orc_set_material(orc_mesh *m, const double *lam_int, const double *mu_int) {
  int mx = 2 * m->nel[0] + 1, my = 2 * m->nel[1] + 1, mz = 2 * m->nel[2] + 1;
  for (int k = 0; k < m->nn[2]; k++)
    for (int j = 0; j < m->nn[1]; j++)
      for (int i = 0; i < m->nn[0]; i++) {
        int ii = i - 2 * m->lo[0], jj = j - 2 * m->lo[1], kk = k - 2 * m->lo[2];
        ii = ii < 0 ? 0 : (ii > mx - 1 ? mx - 1 : ii);
        jj = jj < 0 ? 0 : (jj > my - 1 ? my - 1 : jj);
        kk = kk < 0 ? 0 : (kk > mz - 1 ? mz - 1 : kk);
        long s = ((long)kk * my + jj) * mx + ii;
        long g = node_id(m, i, j, k);
        m->lam[g] = lam_int[s];
        m->mu[g] = mu_int[s];
      }
  return 0;
}

void orc_get_diag(const orc_mesh *m, int which, double *out) {
  const double *src[9] = {m->Mu, m->Cu, m->Ku, m->Gu, m->Ms, m->Cs, m->Ks, m->Gs, m->Mtilde};
  long n = (which == 8) ? m->nmat : m->nnode;
  memcpy(out, src[which], sizeof(double) * n);
}

void orc_get_masks(const orc_mesh *m, unsigned char *pml, unsigned char *dir) {
  memcpy(pml, m->pml_node, m->nnode);
  memcpy(dir, m->dir_node, m->nnode);
}

void orc_get_stretch(const orc_mesh *m, int ax, double *al, double *be) {
  memcpy(al, m->al[ax], sizeof(double) * m->nn[ax]);
  memcpy(be, m->be[ax], sizeof(double) * m->nn[ax]);
}

/* ------------------------------------------------------- element loops
 * Elements are visited in 8 colour classes (parity of ex, ey, ez). Two
 * elements of one class share no node, so the scatter of one class may run
 * in parallel without races, and every node receives its contributions in
 * the same order on every run. */

typedef void (*elem_fn)(const orc_mesh *m, int ex, int ey, int ez, void *ctx);

static void for_elements(const orc_mesh *m, int which, elem_fn fn, void *ctx) {
  /* which: 0 = interior (RD) elements, 1 = PML elements */
  for (int colour = 0; colour < 8; colour++) {
    int px = colour & 1, py = (colour >> 1) & 1, pz = (colour >> 2) & 1;
    int cx = (m->N[0] - px + 1) / 2, cy = (m->N[1] - py + 1) / 2, cz = (m->N[2] - pz + 1) / 2;
    long total = (long)cx * cy * cz;
#pragma omp parallel for schedule(static) num_threads(m->nthreads)
    for (long t = 0; t < total; t++) {
      int ex = px + 2 * (int)(t % cx);
      int ey = py + 2 * (int)((t / cx) % cy);
      int ez = pz + 2 * (int)(t / ((long)cx * cy));
      int rd = elem_is_rd(m, ex, ey, ez);
      if ((which == 0) != (rd != 0)) continue;
      fn(m, ex, ey, ez, ctx);
    }
  }
}

/* gradient G[i][j] = d v_i / d x_j at local quadrature point q of element e,
 * v given per node with stride `st` and offset `off` (components off..off+2) */
static void elem_grad(const orc_mesh *m, int ex, int ey, int ez, const int q[3],
                      const double *v, int st, int off, double G[3][3]) {
  /* d phi_a / d x_j (x_q) vanishes unless a lies on the j-line through q, so
   * the sum over the 27 nodes a runs over those three nodes only */
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) G[i][j] = 0.0;
  for (int j = 0; j < 3; j++)
    for (int b = 0; b < 3; b++) {
      int a[3] = {q[0], q[1], q[2]};
      a[j] = b;
      double dp = dphi(m, a, q, j);
      long g = elem_node(m, ex, ey, ez, a[0], a[1], a[2]);
      for (int i = 0; i < 3; i++) G[i][j] += v[g * st + off + i] * dp;
    }
}

/* ---- K_RD u: int_RD grad(w~) : {mu [grad u + grad u^T] + lambda div u I}  (3a) */
typedef struct { const double *u; double *f; } krd_ctx;

static void krd_elem(const orc_mesh *m, int ex, int ey, int ez, void *vctx) {
  krd_ctx *k = (krd_ctx *)vctx;
  for (int cq = 0; cq < 27; cq++) {
    int q[3] = {cq % 3, (cq / 3) % 3, cq / 9};
    long gq = elem_node(m, ex, ey, ez, q[0], q[1], q[2]);
    double G[3][3], sig[3][3];
    elem_grad(m, ex, ey, ez, q, k->u, 3, 0, G);
    double tr = G[0][0] + G[1][1] + G[2][2];
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++)
        sig[i][j] = m->mu[gq] * (G[i][j] + G[j][i]) + (i == j ? m->lam[gq] * tr : 0.0);
    double wq = quad_weight(m, q);
    for (int j = 0; j < 3; j++)
      for (int b = 0; b < 3; b++) { /* nodes a with d phi_a/dx_j (x_q) != 0 */
        int a[3] = {q[0], q[1], q[2]};
        a[j] = b;
        long ga = elem_node(m, ex, ey, ez, a[0], a[1], a[2]);
        double dp = dphi(m, a, q, j);
        for (int i = 0; i < 3; i++) k->f[ga * 3 + i] += wq * dp * sig[i][j];
      }
  }
}

/* f += K_RD u ; u, f: [nnode][3] */
void orc_apply_KRD(const orc_mesh *m, const double *u, double *f) {
  krd_ctx k = {u, f};
  for_elements(m, 0, krd_elem, &k);
}

/* Lambda tensors at node g: which = 0 (Lambda_e), 1 (Lambda_p), 2 (Lambda_w) */
static void lam_tensor(const orc_mesh *m, long g, int which, double L[3]) {
  double Le[3], Lp[3], Lw[3];
  coef_at(m, g, NULL, NULL, NULL, NULL, Le, Lp, Lw);
  const double *s = which == 0 ? Le : (which == 1 ? Lp : Lw);
  L[0] = s[0]; L[1] = s[1]; L[2] = s[2];
}

/* ---- A_L S (u rows): int_PML grad(w~) : (S^T Lambda)      ((3a), PML term)
 * S symmetric, stored as 6 components; (S^T Lambda)_ij = S_ij Lambda_jj */
typedef struct { int which; const double *in; double *out; } op_ctx;

static void A_elem(const orc_mesh *m, int ex, int ey, int ez, void *vctx) {
  op_ctx *k = (op_ctx *)vctx;
  for (int cq = 0; cq < 27; cq++) {
    int q[3] = {cq % 3, (cq / 3) % 3, cq / 9};
    long gq = elem_node(m, ex, ey, ez, q[0], q[1], q[2]);
    double L[3], Q[3][3];
    lam_tensor(m, gq, k->which, L);
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) Q[i][j] = k->in[gq * 6 + SYM[i][j]] * L[j];
    double wq = quad_weight(m, q);
    for (int j = 0; j < 3; j++)
      for (int b = 0; b < 3; b++) {
        int a[3] = {q[0], q[1], q[2]};
        a[j] = b;
        long ga = elem_node(m, ex, ey, ez, a[0], a[1], a[2]);
        double dp = dphi(m, a, q, j);
        for (int i = 0; i < 3; i++) k->out[ga * 3 + i] += wq * dp * Q[i][j];
      }
  }
}

/* A_L^T w (S rows): the transpose of A_elem's loop, term by term */
static void At_elem(const orc_mesh *m, int ex, int ey, int ez, void *vctx) {
  op_ctx *k = (op_ctx *)vctx;
  for (int cq = 0; cq < 27; cq++) {
    int q[3] = {cq % 3, (cq / 3) % 3, cq / 9};
    long gq = elem_node(m, ex, ey, ez, q[0], q[1], q[2]);
    double L[3];
    lam_tensor(m, gq, k->which, L);
    double wq = quad_weight(m, q);
    for (int j = 0; j < 3; j++)
      for (int b = 0; b < 3; b++) {
        int a[3] = {q[0], q[1], q[2]};
        a[j] = b;
        long ga = elem_node(m, ex, ey, ez, a[0], a[1], a[2]);
        double dp = dphi(m, a, q, j);
        for (int i = 0; i < 3; i++)
          k->out[gq * 6 + SYM[i][j]] += wq * dp * L[j] * k->in[ga * 3 + i];
      }
  }
}

/* ---- B_L u (S rows): int_PML T~ : { mu [(grad u) L + L (grad u)^T]
 *                                   + lambda div(L u) I }        ((3b) right side)
 * div(L u) = sum_k L_kk d u_k / d x_k because L_kk does not depend on x_k. */
static void B_elem(const orc_mesh *m, int ex, int ey, int ez, void *vctx) {
  op_ctx *k = (op_ctx *)vctx;
  for (int cq = 0; cq < 27; cq++) {
    int q[3] = {cq % 3, (cq / 3) % 3, cq / 9};
    long gq = elem_node(m, ex, ey, ez, q[0], q[1], q[2]);
    double L[3], G[3][3];
    lam_tensor(m, gq, k->which, L);
    elem_grad(m, ex, ey, ez, q, k->in, 3, 0, G);
    double dv = G[0][0] * L[0] + G[1][1] * L[1] + G[2][2] * L[2];
    double wq = quad_weight(m, q);
    for (int i = 0; i < 3; i++)
      for (int j = i; j < 3; j++) {
        double R = m->mu[gq] * (G[i][j] * L[j] + L[i] * G[j][i]) + (i == j ? m->lam[gq] * dv : 0.0);
        k->out[gq * 6 + SYM[i][j]] += wq * R;
      }
  }
}

/* B_L^T T (u rows): the transpose of B_elem's loop, term by term */
static void Bt_elem(const orc_mesh *m, int ex, int ey, int ez, void *vctx) {
  op_ctx *k = (op_ctx *)vctx;
  for (int cq = 0; cq < 27; cq++) {
    int q[3] = {cq % 3, (cq / 3) % 3, cq / 9};
    long gq = elem_node(m, ex, ey, ez, q[0], q[1], q[2]);
    double L[3];
    lam_tensor(m, gq, k->which, L);
    double wq = quad_weight(m, q);
    double mu = m->mu[gq], lam = m->lam[gq];
    for (int ca = 0; ca < 27; ca++) {
      int a[3] = {ca % 3, (ca / 3) % 3, ca / 9};
      /* only nodes on a line through q have a nonzero basis gradient at q */
      int off_lines = (a[0] != q[0]) + (a[1] != q[1]) + (a[2] != q[2]);
      if (off_lines > 1) continue;
      long ga = elem_node(m, ex, ey, ez, a[0], a[1], a[2]);
      double dp[3];
      for (int j = 0; j < 3; j++) dp[j] = dphi(m, a, q, j);
      for (int i = 0; i < 3; i++)
        for (int j = i; j < 3; j++) {
          double t = wq * k->in[gq * 6 + SYM[i][j]];
          /* R_ij depends on u_a,i through mu G_ij L_j and on u_a,j through mu L_i G_ji */
          k->out[ga * 3 + i] += t * mu * dp[j] * L[j];
          k->out[ga * 3 + j] += t * mu * L[i] * dp[i];
          if (i == j)
            for (int c = 0; c < 3; c++) k->out[ga * 3 + c] += t * lam * dp[c] * L[c];
        }
    }
  }
}

/* out += op(in). which_L: 0 e, 1 p, 2 w.  A: S[6] -> u[3]; At: u -> S; B: u -> S; Bt: S -> u */
void orc_apply_A(const orc_mesh *m, int which_L, const double *S, double *fu) {
  op_ctx k = {which_L, S, fu};
  for_elements(m, 1, A_elem, &k);
}
void orc_apply_At(const orc_mesh *m, int which_L, const double *w, double *rs) {
  op_ctx k = {which_L, w, rs};
  for_elements(m, 1, At_elem, &k);
}
void orc_apply_B(const orc_mesh *m, int which_L, const double *u, double *rs) {
  op_ctx k = {which_L, u, rs};
  for_elements(m, 1, B_elem, &k);
}
void orc_apply_Bt(const orc_mesh *m, int which_L, const double *T, double *fu) {
  op_ctx k = {which_L, T, fu};
  for_elements(m, 1, Bt_elem, &k);
}

/* ------------------------------------------------------ first-order system */

static void split_level(const orc_mesh *m, const double *lvl, double *u, double *S) {
  for (long g = 0; g < m->nnode; g++) {
    for (int c = 0; c < 3; c++) u[g * 3 + c] = lvl[g * NV + c];
    for (int c = 0; c < 6; c++) S[g * 6 + c] = lvl[g * NV + 3 + c];
  }
}

/* Right-hand side of the first-order system.
 * adjoint = 0: Eq. (6)  d/dt [x0; x1; M x2] = [x1|PML; x2; f - G x0 - K x1 - C x2]
 * adjoint = 1: Eq. (15)/(B.2)  d/dt [y0; y1; M y2] = [y1|PML; y2; G^T y0 - K^T y1 + C^T y2 + f]
 * with the block structure of (3a)/(3b) (and (13a)/(13b) for the adjoint):
 *   u rows: M_uu = rho a, C_uu = rho b, K_uu = rho c + K_RD, G_uu = rho d (lumped),
 *           C_uS = A_e, K_uS = A_p, G_uS = A_w;
 *   S rows: M_SS = a, C_SS = b, K_SS = c, G_SS = d (lumped),
 *           C_Su = -B_e, K_Su = -B_p, G_Su = -B_w.
 * Y, dY: [3][nnode][9]; fext: [nnode][3] nodal point forces, or NULL. */
void orc_rhs(const orc_mesh *m, int adjoint, const double *Y, const double *fext, double *dY) {
  long n = m->nnode;
  double *u[3], *S[3];
  for (int l = 0; l < 3; l++) {
    u[l] = (double *)malloc(sizeof(double) * n * 3);
    S[l] = (double *)malloc(sizeof(double) * n * 6);
    split_level(m, Y + (long)l * n * NV, u[l], S[l]);
  }
  double *fu = (double *)calloc(n * 3, sizeof(double));
  double *rs = (double *)calloc(n * 6, sizeof(double));
  double *tu = (double *)calloc(n * 3, sizeof(double));
  double *ts = (double *)calloc(n * 6, sizeof(double));
  if (!adjoint) {
    /* u rows: f - G x0 - K x1 - C x2 */
    for (long g = 0; g < n; g++)
      for (int c = 0; c < 3; c++)
        fu[g * 3 + c] = (fext ? fext[g * 3 + c] : 0.0) - m->Cu[g] * u[2][g * 3 + c] -
                        m->Ku[g] * u[1][g * 3 + c] - m->Gu[g] * u[0][g * 3 + c];
    orc_apply_KRD(m, u[1], tu);
    orc_apply_A(m, 0, S[2], tu);
    orc_apply_A(m, 1, S[1], tu);
    orc_apply_A(m, 2, S[0], tu);
    for (long i = 0; i < n * 3; i++) fu[i] -= tu[i];
    /* S rows: B_e x2 + B_p x1 + B_w x0 - (b S2 + c S1 + d S0) */
    orc_apply_B(m, 0, u[2], rs);
    orc_apply_B(m, 1, u[1], rs);
    orc_apply_B(m, 2, u[0], rs);
    for (long g = 0; g < n; g++)
      for (int c = 0; c < 6; c++)
        rs[g * 6 + c] -= m->Cs[g] * S[2][g * 6 + c] + m->Ks[g] * S[1][g * 6 + c] +
                         m->Gs[g] * S[0][g * 6 + c];
  } else {
    /* u rows: G^T y0 - K^T y1 + C^T y2 + f */
    for (long g = 0; g < n; g++)
      for (int c = 0; c < 3; c++)
        fu[g * 3 + c] = (fext ? fext[g * 3 + c] : 0.0) + m->Gu[g] * u[0][g * 3 + c] -
                        m->Ku[g] * u[1][g * 3 + c] + m->Cu[g] * u[2][g * 3 + c];
    orc_apply_KRD(m, u[1], tu);          /* K_RD^T = K_RD (pinned by a test) */
    for (long i = 0; i < n * 3; i++) fu[i] -= tu[i];
    memset(tu, 0, sizeof(double) * n * 3);
    orc_apply_Bt(m, 2, S[0], tu);        /* (G_Su)^T y0_S = -B_w^T y0_S */
    for (long i = 0; i < n * 3; i++) fu[i] -= tu[i];
    memset(tu, 0, sizeof(double) * n * 3);
    orc_apply_Bt(m, 1, S[1], tu);        /* -(K_Su)^T y1_S = +B_p^T y1_S */
    for (long i = 0; i < n * 3; i++) fu[i] += tu[i];
    memset(tu, 0, sizeof(double) * n * 3);
    orc_apply_Bt(m, 0, S[2], tu);        /* (C_Su)^T y2_S = -B_e^T y2_S */
    for (long i = 0; i < n * 3; i++) fu[i] -= tu[i];
    /* S rows: (G_uS)^T y0_u + d y0_S - (K_uS)^T y1_u - c y1_S + (C_uS)^T y2_u + b y2_S */
    orc_apply_At(m, 2, u[0], rs);
    orc_apply_At(m, 0, u[2], rs);
    orc_apply_At(m, 1, u[1], ts);
    for (long g = 0; g < n; g++)
      for (int c = 0; c < 6; c++)
        rs[g * 6 + c] += -ts[g * 6 + c] + m->Gs[g] * S[0][g * 6 + c] -
                         m->Ks[g] * S[1][g * 6 + c] + m->Cs[g] * S[2][g * 6 + c];
  }
  double *d0 = dY, *d1 = dY + n * NV, *d2 = dY + 2 * n * NV;
  const double *y1 = Y + n * NV, *y2 = Y + 2 * n * NV;
  for (long g = 0; g < n; g++) {
    int pml = m->pml_node[g], dir = m->dir_node[g];
    for (int c = 0; c < 3; c++) {
      d0[g * NV + c] = (pml && !dir) ? y1[g * NV + c] : 0.0; /* history only in the PML, (5b) */
      d1[g * NV + c] = dir ? 0.0 : y2[g * NV + c];
      d2[g * NV + c] = dir ? 0.0 : fu[g * 3 + c] / m->Mu[g];
    }
    for (int c = 0; c < 6; c++) {
      d0[g * NV + 3 + c] = pml ? y1[g * NV + 3 + c] : 0.0;
      d1[g * NV + 3 + c] = pml ? y2[g * NV + 3 + c] : 0.0;
      d2[g * NV + 3 + c] = pml ? rs[g * 6 + c] / m->Ms[g] : 0.0;
    }
  }
  for (int l = 0; l < 3; l++) { free(u[l]); free(S[l]); }
  free(fu); free(rs); free(tu); free(ts);
}

/* ------------------------------------------------------------- wavelets */

/* kind 0: Ricker  A (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2), tau = t - t0;
 *         params = {f0, t0, A}
 * kind 1: Gaussian pulse of Table 1, read as A exp(-(t - mu)^2 / sigma);
 *         params = {mu, sigma, A} */
double orc_wavelet(int kind, const double *p, double t) {
  if (kind == 0) {
    double a = M_PI * p[0] * (t - p[1]);
    return p[2] * (1.0 - 2.0 * a * a) * exp(-a * a);
  }
  double x = t - p[0];
  return p[2] * exp(-x * x / p[1]);
}

/* ---------------------------------------------------------------- forward */

static void fill_force(const orc_mesh *m, double *fext, int nsrc, const long *node,
                       const double *dir, int kind, const double *wp, double t) {
  memset(fext, 0, sizeof(double) * m->nnode * 3);
  for (int s = 0; s < nsrc; s++) {
    double r = orc_wavelet(kind, wp, t);
    for (int c = 0; c < 3; c++) fext[node[s] * 3 + c] += r * dir[s * 3 + c];
  }
}

static void axpy_state(long n, double *dst, const double *x, double a, const double *y) {
  for (long i = 0; i < n; i++) dst[i] = x[i] + a * y[i];
}

/* Classic RK4 on (6), system initially at rest. Point forces at nodes with
 * direction dir and wavelet (kind, wp). traces[n][r][c] = u_c(x_r, t_n),
 * n = 0..nsteps. uhist (optional): [nsteps+1][nnode][3] displacement history. */
int orc_forward(orc_mesh *m, double dt, int nsteps, int nsrc, const long *src_node,
                const double *src_dir, int kind, const double *wp, int nrec,
                const long *rec_node, double *traces, double *uhist) {
  long n = m->nnode, ns = 3 * n * NV;
  double *X = (double *)calloc(ns, sizeof(double));
  double *T = (double *)malloc(sizeof(double) * ns);
  double *k[4];
  for (int s = 0; s < 4; s++) k[s] = (double *)malloc(sizeof(double) * ns);
  double *fe = (double *)malloc(sizeof(double) * n * 3);
  const double *u = X + n * NV;
  for (int r = 0; r < nrec; r++)
    for (int c = 0; c < 3; c++) traces[r * 3 + c] = 0.0;
  if (uhist) memset(uhist, 0, sizeof(double) * n * 3);
  for (int it = 0; it < nsteps; it++) {
    double t = it * dt;
    fill_force(m, fe, nsrc, src_node, src_dir, kind, wp, t);
    orc_rhs(m, 0, X, fe, k[0]);
    fill_force(m, fe, nsrc, src_node, src_dir, kind, wp, t + 0.5 * dt);
    axpy_state(ns, T, X, 0.5 * dt, k[0]);
    orc_rhs(m, 0, T, fe, k[1]);
    axpy_state(ns, T, X, 0.5 * dt, k[1]);
    orc_rhs(m, 0, T, fe, k[2]);
    fill_force(m, fe, nsrc, src_node, src_dir, kind, wp, t + dt);
    axpy_state(ns, T, X, dt, k[2]);
    orc_rhs(m, 0, T, fe, k[3]);
    for (long i = 0; i < ns; i++)
      X[i] += dt / 6.0 * (k[0][i] + 2.0 * k[1][i] + 2.0 * k[2][i] + k[3][i]);
    for (int r = 0; r < nrec; r++)
      for (int c = 0; c < 3; c++)
        traces[((long)(it + 1) * nrec + r) * 3 + c] = u[rec_node[r] * NV + c];
    if (uhist)
      for (long g = 0; g < n; g++)
        for (int c = 0; c < 3; c++) uhist[((long)(it + 1) * n + g) * 3 + c] = u[g * NV + c];
  }
  free(X); free(T); free(fe);
  for (int s = 0; s < 4; s++) free(k[s]);
  return 0;
}

/* one forward RK4 step of (6) without forcing; Y: [3][nnode][9] in place */
void orc_rk4_step(orc_mesh *m, double *Y, double dt) {
  long ns = 3 * m->nnode * NV;
  double *T = (double *)malloc(sizeof(double) * ns);
  double *k[4];
  for (int s = 0; s < 4; s++) k[s] = (double *)malloc(sizeof(double) * ns);
  orc_rhs(m, 0, Y, NULL, k[0]);
  axpy_state(ns, T, Y, 0.5 * dt, k[0]);
  orc_rhs(m, 0, T, NULL, k[1]);
  axpy_state(ns, T, Y, 0.5 * dt, k[1]);
  orc_rhs(m, 0, T, NULL, k[2]);
  axpy_state(ns, T, Y, dt, k[2]);
  orc_rhs(m, 0, T, NULL, k[3]);
  for (long i = 0; i < ns; i++) Y[i] += dt / 6.0 * (k[0][i] + 2 * k[1][i] + 2 * k[2][i] + k[3][i]);
  free(T);
  for (int s = 0; s < 4; s++) free(k[s]);
}

/* misfit (7) with the trapezoid rule in time (reading R5):
 * J = 1/2 sum_r sum_n w_n dt |u(x_r,t_n) - u_m(x_r,t_n)|^2 */
double orc_misfit(int nsteps, int nrec, double dt, const double *traces, const double *obs) {
  double J = 0.0;
  for (int it = 0; it <= nsteps; it++) {
    double wn = (it == 0 || it == nsteps) ? 0.5 : 1.0;
    double s = 0.0;
    for (long r = 0; r < (long)nrec * 3; r++) {
      double e = traces[(long)it * nrec * 3 + r] - obs[(long)it * nrec * 3 + r];
      s += e * e;
    }
    J += 0.5 * wn * dt * s;
  }
  return J;
}

/* ------------------------------------------------------------- gradient */

typedef struct { const double *u, *w; double wdt; double *gl, *gm; } grad_ctx;

/* (C.1f), (C.1g): at each quadrature point of an interior element,
 * g_lam[i] -= wdt * W detJ * (div w)(div u)
 * g_mu[i]  -= wdt * W detJ * [2(w_x,x u_x,x + w_y,y u_y,y + w_z,z u_z,z)
 *                 + (w_x,y + w_y,x)(u_y,x + u_x,y) + (w_x,z + w_z,x)(u_z,x + u_x,z)
 *                 + (w_y,z + w_z,y)(u_z,y + u_y,z)]
 * chi_i is the nodal basis, so at quadrature point q only chi_q is nonzero. */
static void grad_elem(const orc_mesh *m, int ex, int ey, int ez, void *vctx) {
  grad_ctx *k = (grad_ctx *)vctx;
  int mx = 2 * m->nel[0] + 1, my = 2 * m->nel[1] + 1;
  for (int cq = 0; cq < 27; cq++) {
    int q[3] = {cq % 3, (cq / 3) % 3, cq / 9};
    double Gu[3][3], Gw[3][3];
    elem_grad(m, ex, ey, ez, q, k->u, 3, 0, Gu);
    elem_grad(m, ex, ey, ez, q, k->w, 3, 0, Gw);
    double divw = Gw[0][0] + Gw[1][1] + Gw[2][2];
    double divu = Gu[0][0] + Gu[1][1] + Gu[2][2];
    double gmu = 2.0 * (Gw[0][0] * Gu[0][0] + Gw[1][1] * Gu[1][1] + Gw[2][2] * Gu[2][2]) +
                 (Gw[0][1] + Gw[1][0]) * (Gu[1][0] + Gu[0][1]) +
                 (Gw[0][2] + Gw[2][0]) * (Gu[2][0] + Gu[0][2]) +
                 (Gw[1][2] + Gw[2][1]) * (Gu[2][1] + Gu[1][2]);
    double wq = quad_weight(m, q);
    int mi = 2 * (ex - m->lo[0]) + q[0], mj = 2 * (ey - m->lo[1]) + q[1],
        mk = 2 * (ez - m->lo[2]) + q[2];
    long s = ((long)mk * my + mj) * mx + mi;
    k->gl[s] -= k->wdt * wq * divw * divu;
    k->gm[s] -= k->wdt * wq * gmu;
  }
}

/* Reverse RK4 of Appendix B for (15) (transposes restored, reading R3),
 * driven by the receiver residual e = u - u_m:  f_adj(x_r, t_n) = e^n_r.
 * Half-step forcing: (e^n + e^{n-1}) / 2 (reading R4).
 * Accumulates the misfit gradients (C.1f)/(C.1g) with trapezoid weights (R5).
 * uhist: forward displacement [nsteps+1][nnode][3]; resid: [nsteps+1][nrec][3].
 * g_lam, g_mu: [nmat], overwritten. */
int orc_adjoint_gradient(orc_mesh *m, double dt, int nsteps, int nrec, const long *rec_node,
                         const double *resid, const double *uhist, double *g_lam, double *g_mu) {
  long n = m->nnode, ns = 3 * n * NV;
  double *Y = (double *)calloc(ns, sizeof(double));
  double *T = (double *)malloc(sizeof(double) * ns);
  double *k[4];
  for (int s = 0; s < 4; s++) k[s] = (double *)malloc(sizeof(double) * ns);
  double *fa = (double *)calloc(n * 3, sizeof(double));
  double *w = (double *)malloc(sizeof(double) * n * 3);
  memset(g_lam, 0, sizeof(double) * m->nmat);
  memset(g_mu, 0, sizeof(double) * m->nmat);
#define SET_FORCE(expr)                                              \
  do {                                                               \
    memset(fa, 0, sizeof(double) * n * 3);                           \
    for (int r = 0; r < nrec; r++)                                   \
      for (int c = 0; c < 3; c++) fa[rec_node[r] * 3 + c] += (expr); \
  } while (0)
#define RES(it) resid[((long)(it) * nrec + r) * 3 + c]
  for (int it = nsteps; it >= 1; it--) {
    SET_FORCE(RES(it));
    orc_rhs(m, 1, Y, fa, k[0]);
    SET_FORCE(0.5 * (RES(it) + RES(it - 1)));
    axpy_state(ns, T, Y, -0.5 * dt, k[0]);
    orc_rhs(m, 1, T, fa, k[1]);
    axpy_state(ns, T, Y, -0.5 * dt, k[1]);
    orc_rhs(m, 1, T, fa, k[2]);
    SET_FORCE(RES(it - 1));
    axpy_state(ns, T, Y, -dt, k[2]);
    orc_rhs(m, 1, T, fa, k[3]);
    for (long i = 0; i < ns; i++)
      Y[i] -= dt / 6.0 * (k[0][i] + 2.0 * k[1][i] + 2.0 * k[2][i] + k[3][i]);
    /* adjoint displacement at t_{it-1} */
    for (long g = 0; g < n; g++)
      for (int c = 0; c < 3; c++) w[g * 3 + c] = Y[n * NV + g * NV + c];
    int lvl = it - 1;
    double wn = (lvl == 0 || lvl == nsteps) ? 0.5 : 1.0;
    grad_ctx gc = {uhist + (long)lvl * n * 3, w, wn * dt, g_lam, g_mu};
    for_elements(m, 0, grad_elem, &gc);
  }
#undef SET_FORCE
#undef RES
  free(Y); free(T); free(fa); free(w);
  for (int s = 0; s < 4; s++) free(k[s]);
  return 0;
}

/* one-time-level gradient integrand with weight wdt (exported for tests) */
void orc_gradient_term(orc_mesh *m, const double *u, const double *w, double wdt,
                       double *g_lam, double *g_mu) {
  grad_ctx gc = {u, w, wdt, g_lam, g_mu};
  for_elements(m, 0, grad_elem, &gc);
}

/* kinetic and interior strain energy of a state Y: [3][nnode][9]
 * out[0] = 1/2 v^T M_uu v, out[1] = 1/2 u^T K_RD u */
void orc_energy(orc_mesh *m, const double *Y, double *out) {
  long n = m->nnode;
  const double *y1 = Y + n * NV, *y2 = Y + 2 * n * NV;
  double *u = (double *)malloc(sizeof(double) * n * 3);
  double *f = (double *)calloc(n * 3, sizeof(double));
  double ek = 0.0, es = 0.0;
  for (long g = 0; g < n; g++)
    for (int c = 0; c < 3; c++) {
      u[g * 3 + c] = y1[g * NV + c];
      ek += 0.5 * m->Mu[g] * y2[g * NV + c] * y2[g * NV + c];
    }
  orc_apply_KRD(m, u, f);
  for (long i = 0; i < n * 3; i++) es += 0.5 * u[i] * f[i];
  out[0] = ek; out[1] = es;
  free(u); free(f);
}

/* ---- regularisation, Sec. 3.1 Eqs. (8)/(9), gradients (C.1b)-(C.1e).
 * f: a nodal field on the interior (material) grid [nmat], e.g. lambda or mu.
 * For every interior element and quadrature point q (the element's 27 nodes):
 *   grad f_h(q) from the element's nodal values (chi = the nodal Lagrange basis),
 *   TN (kind 0): R += W detJ |grad f_h(q)|^2 / 2,
 *                g_a += W detJ grad chi_a(q) . grad f_h(q)                  (C.1b/c)
 *   TV (kind 1): R += W detJ (|grad f_h(q)|^2 + eps)^(1/2),
 *                g_a += W detJ grad chi_a(q) . grad f_h(q) / (|grad f_h(q)|^2 + eps)^(1/2)
 *                                                                  (C.1d/e, R8)
 * without the factors R_lambda, R_mu. Plain serial element loop. g is overwritten. */
static long mat_node_of(const orc_mesh *m, int ex, int ey, int ez, const int a[3]) {
  int mx = 2 * m->nel[0] + 1, my = 2 * m->nel[1] + 1;
  int i = 2 * (ex - m->lo[0]) + a[0], j = 2 * (ey - m->lo[1]) + a[1], k = 2 * (ez - m->lo[2]) + a[2];
  return ((long)k * my + j) * mx + i;
}

double orc_regularization(const orc_mesh *m, int kind, double eps, const double *f, double *g) {
  memset(g, 0, sizeof(double) * m->nmat);
  double R = 0.0;
  for (int ez = m->lo[2]; ez < m->hi[2]; ez++)
    for (int ey = m->lo[1]; ey < m->hi[1]; ey++)
      for (int ex = m->lo[0]; ex < m->hi[0]; ex++)
        for (int cq = 0; cq < 27; cq++) {
          int q[3] = {cq % 3, (cq / 3) % 3, cq / 9};
          double gf[3] = {0.0, 0.0, 0.0};
          for (int j = 0; j < 3; j++)
            for (int b = 0; b < 3; b++) {
              int a[3] = {q[0], q[1], q[2]};
              a[j] = b;
              gf[j] += dphi(m, a, q, j) * f[mat_node_of(m, ex, ey, ez, a)];
            }
          double s2 = gf[0] * gf[0] + gf[1] * gf[1] + gf[2] * gf[2];
          double wq = quad_weight(m, q);
          double scale = 1.0;
          if (kind == 1) {
            double root = sqrt(s2 + eps);
            R += wq * root;
            scale = 1.0 / root;
          } else {
            R += 0.5 * wq * s2;
          }
          for (int j = 0; j < 3; j++)
            for (int b = 0; b < 3; b++) {
              int a[3] = {q[0], q[1], q[2]};
              a[j] = b;
              g[mat_node_of(m, ex, ey, ez, a)] += wq * dphi(m, a, q, j) * gf[j] * scale;
            }
        }
  return R;
}
