/*
 * fnn_oracle.c -- plain, slow, float64 reference for the ANI-style energy path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product links or calls this file;
 * only the test-suite, the smoke check and the benchmark's CPU-baseline leg do.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (FeNNol, arXiv 2405.01491):
 *   - oracle_neighbors : the directed neighbour graph of section II.A
 *     ("GraphGenerator"): all pairs (i, j), i != j, of the same structure with
 *     distance below the cutoff, each unordered pair twice, with the integer
 *     image shift n (minimum image convention) when the structure is periodic.
 *     It is the paper's own all-pairs algorithm (section II.A), written out.
 *   - oracle_aev       : the ANI atomic environment vector named in sections
 *     II.B and II.E (Fig. ani_diagram): Gaussian radial basis (section II.B)
 *     times the cosine switching function (section II.A, processing modules),
 *     and the ANI angular term over unordered pairs of neighbours {jk}
 *     (Appendix A, angular resources, with Theta_n of ANI).  The ANI-2x
 *     constants and the parts the paper leaves unstated are the readings
 *     listed in the design notes (prefactors 1/4 and 2, cos damping 0.95,
 *     shift grids, slot order).
 *   - oracle_aev_vjp   : dE/dx from dE/dAEV by the chain rule (the paper gets
 *     it from jax.grad, section II.E), plus the virial -sum d (x) dE/dd.
 *   - oracle_aev_jvp   : the tangent of the AEV along a displacement field.
 *
 * Conventions: positions double [N][3] and cells double [n_mol][9] (row vectors,
 * orthorhombic only: off-diagonals must be zero).  The shared inputs are float32
 * and are widened exactly by the caller; finite-difference pins perturb them in
 * double.
 * pbc[m] = 1 selects the minimum image convention for molecule m.
 * For an edge (i, j, n): d = (x_j - x_i) + n * L per axis, evaluated in IEEE
 * double with round-to-nearest and no contraction (build with
 * -ffp-contract=off), d2 = (dx*dx + dy*dy) + dz*dz, member iff d2 < R*R.
 * Element order: H C N O F S Cl (Z = 1 6 7 8 9 16 17).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NE 7        /* elements */
#define NSR 16      /* radial shifts */
#define NSA 8       /* angular radial shifts */
#define NSZ 4       /* angular sections */
#define NRAD (NE * NSR)                 /* 112 */
#define NPAIR (NE * (NE + 1) / 2)       /* 28 */
#define NANG (NPAIR * NSA * NSZ)        /* 896 */
#define NAEV (NRAD + NANG)              /* 1008 */

typedef struct {
  double rc_rad, rc_ang;     /* cutoffs, A */
  double eta_r, eta_a, zeta; /* Gaussian widths and angular exponent */
  double shf_r0, shf_a0;     /* first radial / angular-radial shift, A */
  double sw_kind;            /* switching function: 0 cosine, 1 polynomial envelope, 2 exponential */
  double sw_p;               /* exponent p of the polynomial envelope */
} oracle_params;

static const double PI = 3.14159265358979323846;

int oracle_element(int32_t z) {
  switch (z) {
    case 1: return 0; case 6: return 1; case 7: return 2; case 8: return 3;
    case 9: return 4; case 16: return 5; case 17: return 6;
    default: return -1;
  }
}

/* index of the unordered element pair (a, b), a <= b, in row-major upper-triangle order */
static int pair_index(int a, int b) {
  if (a > b) { int t = a; a = b; b = t; }
  return a * NE - a * (a - 1) / 2 + (b - a);
}

/*
 * Switching functions and their derivatives (section II.A processing modules: the cosine function of
 * the ANI models, the polynomial envelope of Gasteiger et al. 2020 and the exponential function of
 * SpookyNet), all 0 from the cutoff on:
 *   cosine:       f = cos(pi r / rc) / 2 + 1/2
 *   polynomial:   f = 1 - (p+1)(p+2)/2 d^p + p(p+2) d^(p+1) - p(p+1)/2 d^(p+2),  d = r / rc
 *   exponential:  f = exp(-r^2 / ((rc - r)(rc + r)))
 */
static int g_sw_kind = 0;     /* set from the parameters at each entry point */
static double g_sw_p = 6.0;
static void set_switch(const void *params) {
  const oracle_params *P = (const oracle_params *)params;
  g_sw_kind = (int)P->sw_kind;
  g_sw_p = P->sw_p;
}
static double fcut(double r, double rc) {
  if (!(r < rc)) return 0.0;
  if (g_sw_kind == 1) {
    double p = g_sw_p, d = r / rc;
    return 1.0 - 0.5 * (p + 1.0) * (p + 2.0) * pow(d, p) + p * (p + 2.0) * pow(d, p + 1.0) -
           0.5 * p * (p + 1.0) * pow(d, p + 2.0);
  }
  if (g_sw_kind == 2) return exp(-r * r / ((rc - r) * (rc + r)));
  return 0.5 * cos(PI * r / rc) + 0.5;
}
static double dfcut(double r, double rc) {
  if (!(r < rc)) return 0.0;
  if (g_sw_kind == 1) {
    double p = g_sw_p, d = r / rc;
    return (-0.5 * p * (p + 1.0) * (p + 2.0) * pow(d, p - 1.0) + p * (p + 1.0) * (p + 2.0) * pow(d, p) -
            0.5 * p * (p + 1.0) * (p + 2.0) * pow(d, p + 1.0)) / rc;
  }
  if (g_sw_kind == 2) {
    double q = (rc - r) * (rc + r);
    return -exp(-r * r / q) * 2.0 * r * rc * rc / (q * q);
  }
  return -0.5 * PI / rc * sin(PI * r / rc);
}

/* the switching function of the given parameters at r (value and derivative), for the pins */
void oracle_switch(const void *params, double r, double rc, double *f, double *df) {
  set_switch(params);
  *f = fcut(r, rc);
  *df = dfcut(r, rc);
}

static int box_of(const double *cell, const uint8_t *pbc, int m, double L[3]) {
  if (!pbc || !pbc[m] || !cell) { L[0] = L[1] = L[2] = 0.0; return 0; }
  const double *c = cell + 9 * (size_t)m;
  if (c[1] != 0.0 || c[2] != 0.0 || c[3] != 0.0 || c[5] != 0.0 || c[6] != 0.0 || c[7] != 0.0) return -1;
  L[0] = c[0]; L[1] = c[4]; L[2] = c[8];
  return 1;
}

/* minimum-image shift and separation for one ordered pair */
static double pair_sep(const double *pos, int i, int j, int periodic, const double L[3], int n[3], double d[3]) {
  for (int a = 0; a < 3; a++) {
    double raw = pos[3 * (size_t)j + a] - pos[3 * (size_t)i + a];
    n[a] = periodic ? -(int)nearbyint(raw / L[a]) : 0;
    d[a] = raw + (double)n[a] * L[a];
  }
  return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
}

/*
 * All directed pairs within R.  Returns the number of pairs (entries beyond
 * cap are not written; call again with a larger cap), or -3 when a periodic
 * cell is not orthorhombic or has an edge <= 2R, -1 on bad arguments.
 * Output order: by i, then by j.
 */
int64_t oracle_neighbors(int32_t n_atoms, int32_t n_mol, const int32_t *mol_offsets, const double *pos,
                         const double *cell, const uint8_t *pbc, double R, int64_t cap,
                         int32_t *out_i, int32_t *out_j, int8_t *out_shift) {
  if (n_atoms < 0 || n_mol < 0 || !mol_offsets) return -1;
  const double R2 = R * R;
  int64_t *cnt = (int64_t *)calloc((size_t)n_atoms + 1, sizeof(int64_t));
  if (!cnt) return -1;
  for (int m = 0; m < n_mol; m++) {
    double L[3];
    int per = box_of(cell, pbc, m, L);
    if (per < 0) { free(cnt); return -3; }
    if (per && (L[0] <= 2 * R || L[1] <= 2 * R || L[2] <= 2 * R)) { free(cnt); return -3; }
  }
  /* pass 1: count per row */
  for (int m = 0; m < n_mol; m++) {
    double L[3];
    int per = box_of(cell, pbc, m, L);
    int a0 = mol_offsets[m], a1 = mol_offsets[m + 1];
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = a0; i < a1; i++) {
      int64_t c = 0;
      for (int j = a0; j < a1; j++) {
        if (j == i) continue;
        int n[3]; double d[3];
        if (pair_sep(pos, i, j, per, L, n, d) < R2) c++;
      }
      cnt[i + 1] = c;
    }
  }
  for (int i = 0; i < n_atoms; i++) cnt[i + 1] += cnt[i];
  int64_t total = cnt[n_atoms];
  if (total <= cap && out_i && out_j) {
    for (int m = 0; m < n_mol; m++) {
      double L[3];
      int per = box_of(cell, pbc, m, L);
      int a0 = mol_offsets[m], a1 = mol_offsets[m + 1];
#pragma omp parallel for schedule(dynamic, 16)
      for (int i = a0; i < a1; i++) {
        int64_t w = cnt[i];
        for (int j = a0; j < a1; j++) {
          if (j == i) continue;
          int n[3]; double d[3];
          if (pair_sep(pos, i, j, per, L, n, d) < R2) {
            out_i[w] = i; out_j[w] = j;
            if (out_shift) for (int a = 0; a < 3; a++) out_shift[3 * w + a] = (int8_t)n[a];
            w++;
          }
        }
      }
    }
  }
  free(cnt);
  return total;
}

/* ----------------------------------------------------------------------------------------- AEV */

typedef struct {
  int32_t n_atoms, n_mol;
  const int32_t *mol_offsets, *Z;
  const double *pos, *cell;
  const uint8_t *pbc;
  int64_t nnz;                      /* edges of the rc_rad graph, sorted by i */
  const int32_t *ei, *ej;
  const int8_t *es;
} oracle_graph;

/* separation vector of an edge, recomputed from coordinates (processing modules, section II.A) */
static void edge_vec(const oracle_graph *g, const int32_t *atom_mol, int64_t e, double d[3]) {
  int i = g->ei[e], j = g->ej[e];
  double L[3];
  box_of(g->cell, g->pbc, atom_mol[i], L);
  for (int a = 0; a < 3; a++)
    d[a] = (g->pos[3 * (size_t)j + a] - g->pos[3 * (size_t)i + a]) + (double)g->es[3 * e + a] * L[a];
}

static int32_t *make_atom_mol(const oracle_graph *g) {
  int32_t *am = (int32_t *)malloc(sizeof(int32_t) * ((size_t)g->n_atoms + 1));
  for (int m = 0; m < g->n_mol; m++)
    for (int i = g->mol_offsets[m]; i < g->mol_offsets[m + 1]; i++) am[i] = m;
  return am;
}

static int64_t *make_row_start(const oracle_graph *g) {
  int64_t *rs = (int64_t *)calloc((size_t)g->n_atoms + 1, sizeof(int64_t));
  for (int64_t e = 0; e < g->nnz; e++) rs[g->ei[e] + 1]++;
  for (int i = 0; i < g->n_atoms; i++) rs[i + 1] += rs[i];
  return rs;
}

/*
 * Per-triplet quantities of the angular term for centre i and neighbours j, k:
 *   c = cos(theta_ijk), theta' = acos(0.95 c),
 *   A_s = ((1 + cos(theta' - theta_s)) / 2)^zeta,  theta_s = pi/8 + s pi/4,
 *   B_m = exp(-eta_a ((r_ij + r_ik)/2 - a_m)^2),    a_m = shf_a0 + m (rc_ang - shf_a0)/8,
 *   C   = fc(r_ij) fc(r_ik);   term[m][s] = 2 A_s B_m C.
 * With want_d, also the partials of every term with respect to r_ij, r_ik and c.
 */
typedef struct { double t[NSA][NSZ], dr1[NSA][NSZ], dr2[NSA][NSZ], dc[NSA][NSZ]; } triplet_terms;

static void angular_terms(const oracle_params *P, double r1, double r2, double c, int want_d, triplet_terms *T) {
  double cp = 0.95 * c;
  double th = acos(cp);
  double dth_dc = -0.95 / sqrt(1.0 - cp * cp);
  double f1 = fcut(r1, P->rc_ang), f2 = fcut(r2, P->rc_ang);
  double C = f1 * f2, dC1 = dfcut(r1, P->rc_ang) * f2, dC2 = f1 * dfcut(r2, P->rc_ang);
  double rbar = 0.5 * (r1 + r2);
  for (int m = 0; m < NSA; m++) {
    double am = P->shf_a0 + m * (P->rc_ang - P->shf_a0) / NSA;
    double B = exp(-P->eta_a * (rbar - am) * (rbar - am));
    double dB_dr = B * (-2.0 * P->eta_a * (rbar - am)) * 0.5; /* same for r1 and r2 */
    for (int s = 0; s < NSZ; s++) {
      double ts = PI / 8.0 + s * PI / 4.0;
      double base = 0.5 * (1.0 + cos(th - ts));
      double A = pow(base, P->zeta);
      T->t[m][s] = 2.0 * A * B * C;
      if (want_d) {
        double dA_dth = P->zeta * pow(base, P->zeta - 1.0) * (-0.5 * sin(th - ts));
        T->dc[m][s] = 2.0 * dA_dth * dth_dc * B * C;
        T->dr1[m][s] = 2.0 * A * (dB_dr * C + B * dC1);
        T->dr2[m][s] = 2.0 * A * (dB_dr * C + B * dC2);
      }
    }
  }
}

static void radial_terms(const oracle_params *P, double r, double t[NSR], double dt[NSR]) {
  double f = fcut(r, P->rc_rad), df = dfcut(r, P->rc_rad);
  for (int k = 0; k < NSR; k++) {
    double rk = P->shf_r0 + k * (P->rc_rad - P->shf_r0) / NSR;
    double gk = exp(-P->eta_r * (r - rk) * (r - rk));
    t[k] = 0.25 * gk * f;
    if (dt) dt[k] = 0.25 * gk * (-2.0 * P->eta_r * (r - rk) * f + df);
  }
}

/* neighbours of centre i inside rc_ang, as edge indices */
static int angular_list(const oracle_graph *g, const oracle_params *P, const int32_t *am, const int64_t *rs,
                        int i, int64_t *out, int cap) {
  int n = 0;
  for (int64_t e = rs[i]; e < rs[i + 1]; e++) {
    double d[3];
    edge_vec(g, am, e, d);
    double r = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
    if (r < P->rc_ang) {
      if (n < cap) out[n] = e;
      n++;
    }
  }
  return n; /* callers treat n > cap as an error */
}

/* Returns 0, or -2 when a species is outside the element table. */
int oracle_aev(const oracle_graph *g, const oracle_params *P, double *aev) {
  set_switch(P);
  int overflow = 0;
  for (int i = 0; i < g->n_atoms; i++) if (oracle_element(g->Z[i]) < 0) return -2;
  int32_t *am = make_atom_mol(g);
  int64_t *rs = make_row_start(g);
  memset(aev, 0, sizeof(double) * NAEV * (size_t)g->n_atoms);
#pragma omp parallel for schedule(dynamic, 8)
  for (int i = 0; i < g->n_atoms; i++) {
    double *out = aev + (size_t)NAEV * i;
    for (int64_t e = rs[i]; e < rs[i + 1]; e++) {
      double d[3], t[NSR];
      edge_vec(g, am, e, d);
      double r = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
      if (!(r < P->rc_rad)) continue;
      radial_terms(P, r, t, NULL);
      int ej = oracle_element(g->Z[g->ej[e]]);
      for (int k = 0; k < NSR; k++) out[ej * NSR + k] += t[k];
    }
    int64_t nb[1024];
    int na = angular_list(g, P, am, rs, i, nb, 1024);
    if (na > 1024) { overflow = 1; na = 1024; }
    for (int a = 0; a < na; a++)
      for (int b = a + 1; b < na; b++) {
        double d1[3], d2[3];
        edge_vec(g, am, nb[a], d1);
        edge_vec(g, am, nb[b], d2);
        double r1 = sqrt((d1[0] * d1[0] + d1[1] * d1[1]) + d1[2] * d1[2]);
        double r2 = sqrt((d2[0] * d2[0] + d2[1] * d2[1]) + d2[2] * d2[2]);
        double c = ((d1[0] * d2[0] + d1[1] * d2[1]) + d1[2] * d2[2]) / (r1 * r2);
        triplet_terms T;
        angular_terms(P, r1, r2, c, 0, &T);
        int p = pair_index(oracle_element(g->Z[g->ej[nb[a]]]), oracle_element(g->Z[g->ej[nb[b]]]));
        double *slot = out + NRAD + p * NSA * NSZ;
        for (int m = 0; m < NSA; m++)
          for (int s = 0; s < NSZ; s++) slot[m * NSZ + s] += T.t[m][s];
      }
  }
  free(am); free(rs);
  return overflow ? -4 : 0;
}

/*
 * Vector-Jacobian product: given G = dE/dAEV [N][1008], writes grad = dE/dx [N][3]
 * and, when virial != NULL, W[m] = -sum over edges of molecule m of d (x) dE/dd
 * (row-major 3x3), which equals sum_i x_i (x) F_i for a gas-phase molecule.
 * Per-edge gradients are formed per centre atom, then scattered serially.
 */
int oracle_aev_vjp(const oracle_graph *g, const oracle_params *P, const double *G, double *grad, double *virial) {
  set_switch(P);
  int overflow = 0;
  for (int i = 0; i < g->n_atoms; i++) if (oracle_element(g->Z[i]) < 0) return -2;
  int32_t *am = make_atom_mol(g);
  int64_t *rs = make_row_start(g);
  double *ge = (double *)calloc((size_t)g->nnz * 3 + 1, sizeof(double)); /* dE/dd per edge */
#pragma omp parallel for schedule(dynamic, 8)
  for (int i = 0; i < g->n_atoms; i++) {
    const double *Gi = G + (size_t)NAEV * i;
    for (int64_t e = rs[i]; e < rs[i + 1]; e++) {
      double d[3], t[NSR], dt[NSR];
      edge_vec(g, am, e, d);
      double r = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
      if (!(r < P->rc_rad)) continue;
      radial_terms(P, r, t, dt);
      int ej = oracle_element(g->Z[g->ej[e]]);
      double dEdr = 0.0;
      for (int k = 0; k < NSR; k++) dEdr += Gi[ej * NSR + k] * dt[k];
      for (int a = 0; a < 3; a++) ge[3 * e + a] += dEdr * d[a] / r;
    }
    int64_t nb[1024];
    int na = angular_list(g, P, am, rs, i, nb, 1024);
    if (na > 1024) { overflow = 1; na = 1024; }
    for (int a = 0; a < na; a++)
      for (int b = a + 1; b < na; b++) {
        double d1[3], d2[3];
        edge_vec(g, am, nb[a], d1);
        edge_vec(g, am, nb[b], d2);
        double r1 = sqrt((d1[0] * d1[0] + d1[1] * d1[1]) + d1[2] * d1[2]);
        double r2 = sqrt((d2[0] * d2[0] + d2[1] * d2[1]) + d2[2] * d2[2]);
        double c = ((d1[0] * d2[0] + d1[1] * d2[1]) + d1[2] * d2[2]) / (r1 * r2);
        triplet_terms T;
        angular_terms(P, r1, r2, c, 1, &T);
        int p = pair_index(oracle_element(g->Z[g->ej[nb[a]]]), oracle_element(g->Z[g->ej[nb[b]]]));
        const double *Gs = Gi + NRAD + p * NSA * NSZ;
        double eR1 = 0, eR2 = 0, eC = 0;
        for (int m = 0; m < NSA; m++)
          for (int s = 0; s < NSZ; s++) {
            eR1 += Gs[m * NSZ + s] * T.dr1[m][s];
            eR2 += Gs[m * NSZ + s] * T.dr2[m][s];
            eC += Gs[m * NSZ + s] * T.dc[m][s];
          }
        /* dc/dd1 = d2/(r1 r2) - c d1/r1^2 ; dr1/dd1 = d1/r1 (and symmetric for d2) */
        for (int x = 0; x < 3; x++) {
          double g1 = eR1 * d1[x] / r1 + eC * (d2[x] / (r1 * r2) - c * d1[x] / (r1 * r1));
          double g2 = eR2 * d2[x] / r2 + eC * (d1[x] / (r1 * r2) - c * d2[x] / (r2 * r2));
          ge[3 * nb[a] + x] += g1;
          ge[3 * nb[b] + x] += g2;
        }
      }
  }
  memset(grad, 0, sizeof(double) * 3 * (size_t)g->n_atoms);
  if (virial) memset(virial, 0, sizeof(double) * 9 * (size_t)g->n_mol);
  for (int64_t e = 0; e < g->nnz; e++) {
    int i = g->ei[e], j = g->ej[e];
    double d[3];
    edge_vec(g, am, e, d);
    for (int a = 0; a < 3; a++) {
      grad[3 * (size_t)j + a] += ge[3 * e + a];
      grad[3 * (size_t)i + a] -= ge[3 * e + a];
    }
    if (virial) {
      double *W = virial + 9 * (size_t)am[i];
      for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) W[3 * a + b] -= d[a] * ge[3 * e + b];
    }
  }
  free(ge); free(am); free(rs);
  return overflow ? -4 : 0;
}

/*
 * Jacobian-vector product: T = (dAEV/dx) . V for a displacement field V [N][3]
 * (directional derivative of every AEV entry).  Used for the force-loss
 * weight gradient: d/dtheta <T, dE/dAEV(theta)>.
 */
int oracle_aev_jvp(const oracle_graph *g, const oracle_params *P, const double *V, double *T_out) {
  set_switch(P);
  int overflow = 0;
  for (int i = 0; i < g->n_atoms; i++) if (oracle_element(g->Z[i]) < 0) return -2;
  int32_t *am = make_atom_mol(g);
  int64_t *rs = make_row_start(g);
  memset(T_out, 0, sizeof(double) * NAEV * (size_t)g->n_atoms);
#pragma omp parallel for schedule(dynamic, 8)
  for (int i = 0; i < g->n_atoms; i++) {
    double *out = T_out + (size_t)NAEV * i;
    for (int64_t e = rs[i]; e < rs[i + 1]; e++) {
      double d[3], t[NSR], dt[NSR], vd[3];
      edge_vec(g, am, e, d);
      double r = sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]);
      if (!(r < P->rc_rad)) continue;
      radial_terms(P, r, t, dt);
      int j = g->ej[e];
      for (int a = 0; a < 3; a++) vd[a] = V[3 * (size_t)j + a] - V[3 * (size_t)i + a];
      double rdot = (d[0] * vd[0] + d[1] * vd[1] + d[2] * vd[2]) / r;
      int ej = oracle_element(g->Z[j]);
      for (int k = 0; k < NSR; k++) out[ej * NSR + k] += dt[k] * rdot;
    }
    int64_t nb[1024];
    int na = angular_list(g, P, am, rs, i, nb, 1024);
    if (na > 1024) { overflow = 1; na = 1024; }
    for (int a = 0; a < na; a++)
      for (int b = a + 1; b < na; b++) {
        double d1[3], d2[3], v1[3], v2[3];
        edge_vec(g, am, nb[a], d1);
        edge_vec(g, am, nb[b], d2);
        int j = g->ej[nb[a]], k = g->ej[nb[b]];
        for (int x = 0; x < 3; x++) {
          v1[x] = V[3 * (size_t)j + x] - V[3 * (size_t)i + x];
          v2[x] = V[3 * (size_t)k + x] - V[3 * (size_t)i + x];
        }
        double r1 = sqrt((d1[0] * d1[0] + d1[1] * d1[1]) + d1[2] * d1[2]);
        double r2 = sqrt((d2[0] * d2[0] + d2[1] * d2[1]) + d2[2] * d2[2]);
        double c = ((d1[0] * d2[0] + d1[1] * d2[1]) + d1[2] * d2[2]) / (r1 * r2);
        double r1dot = 0, r2dot = 0, cdot = 0;
        for (int x = 0; x < 3; x++) {
          r1dot += d1[x] * v1[x] / r1;
          r2dot += d2[x] * v2[x] / r2;
          cdot += (d2[x] / (r1 * r2) - c * d1[x] / (r1 * r1)) * v1[x] + (d1[x] / (r1 * r2) - c * d2[x] / (r2 * r2)) * v2[x];
        }
        triplet_terms TT;
        angular_terms(P, r1, r2, c, 1, &TT);
        int p = pair_index(oracle_element(g->Z[j]), oracle_element(g->Z[k]));
        double *slot = out + NRAD + p * NSA * NSZ;
        for (int m = 0; m < NSA; m++)
          for (int s = 0; s < NSZ; s++)
            slot[m * NSZ + s] += TT.dr1[m][s] * r1dot + TT.dr2[m][s] * r2dot + TT.dc[m][s] * cdot;
      }
  }
  free(am); free(rs);
  return overflow ? -4 : 0;
}
