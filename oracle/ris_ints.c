/*
 * TDDFT-ris oracle: plain FP64 Gaussian integrals on the CPU.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU baseline
 * leg of the benchmark use it.  It shares no code with the CUDA library.
 *
 * What it computes (all over uncontracted, normalised cartesian primitives):
 *   - the three-centre Coulomb integrals (mu nu|P) and the two-centre metric
 *     (P|Q) that the ris kernel of Eq. (g_modified) (Sec. 2.2) is built from;
 *   - their first derivatives with respect to the coordinates of one atom,
 *     each centre differentiated directly (no translational-invariance
 *     shortcut), as needed by the RI derivative formula at the end of
 *     Sec. 2.2;
 *   - the AO overlap and the Boys function, for the pins.
 *
 * Method: Obara-Saika vertical recurrence on [e0|f]^(m) followed by the
 * horizontal transfer (a,b+1_i| = (a+1_i,b| + AB_i (a,b|.  The Boys
 * function uses its defining series for T < 35 and erf + upward recursion
 * beyond.  Derivatives of a primitive use
 *   d/dA_i x_A^{a_i} e^{-alpha r_A^2} = 2 alpha x_A^{a_i+1}... - a_i x_A^{a_i-1}...
 * Plain loops, OpenMP over shell pairs; no screening.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define LMAX_TOT 14

static int nm_upto(int L) { return L < 0 ? 0 : (L + 1) * (L + 2) * (L + 3) / 6; }
static int ncart_l(int l) { return (l + 1) * (l + 2) / 2; }
static int mono_idx(int lx, int ly, int lz) {
  int L = lx + ly + lz;
  return L * (L + 1) * (L + 2) / 6 + (L - lx) * (L - lx + 1) / 2 + lz;
}
/* monomial exponents of flat index k */
static int MX[1024], MY[1024], MZ[1024];
static int tables_ready = 0;
static void init_tables(void) {
  if (tables_ready) return;
  for (int L = 0; L <= LMAX_TOT; L++)
    for (int lx = L; lx >= 0; lx--)
      for (int ly = L - lx; ly >= 0; ly--) {
        int lz = L - lx - ly;
        int k = mono_idx(lx, ly, lz);
        MX[k] = lx; MY[k] = ly; MZ[k] = lz;
      }
  tables_ready = 1;
}
static int comp(int k, int d) { return d == 0 ? MX[k] : (d == 1 ? MY[k] : MZ[k]); }

static double dfact(int n) { /* (2n-1)!! */
  double r = 1.0;
  for (int k = 1; k < 2 * n; k += 2) r *= k;
  return r;
}
static double cart_norm(int lx, int ly, int lz, double a) {
  int L = lx + ly + lz;
  return sqrt(pow(2.0 * a / M_PI, 1.5) * pow(4.0 * a, L) / (dfact(lx) * dfact(ly) * dfact(lz)));
}

double oracle_boys(int m, double T) {
  if (T < 1e-300) return 1.0 / (2 * m + 1);
  if (T < 35.0) {
    double term = 1.0 / (2 * m + 1), sum = term;
    for (int k = 1; k < 2000; k++) {
      term *= 2.0 * T / (2 * m + 2 * k + 1);
      sum += term;
      if (term < 1e-18 * sum) break;
    }
    return exp(-T) * sum;
  }
  double f = 0.5 * sqrt(M_PI / T) * erf(sqrt(T));
  double e = exp(-T);
  for (int k = 0; k < m; k++) f = ((2 * k + 1) * f - e) / (2.0 * T);
  return f;
}

/*
 * Raw (unnormalised) primitive integrals (a b|c) for shells of total
 * angular momenta la, lb, lc; out[ia][ib][ic] over cartesian components in
 * lexicographic order.  beta = 0 with B = A turns this into the two-centre
 * integral (a|c).  scratch must hold at least scratch_size(la,lb,lc).
 */
static size_t scratch_size(int la, int lb, int lc) {
  int Le = la + lb, Lf = lc, M = Le + Lf;
  size_t v = (size_t)(M + 1) * nm_upto(Le) * nm_upto(Lf);
  size_t h = (size_t)nm_upto(Le) * nm_upto(lb) * nm_upto(Lf);
  return v + h + 64;
}

static void prim3c(int la, int lb, int lc, double alpha, const double* A, double beta,
                   const double* B, double gamma, const double* Cc, double* out,
                   double* scratch) {
  const int Le = la + lb, Lf = lc, M = Le + Lf;
  const int NE = nm_upto(Le), NF = nm_upto(Lf);
  double* V = scratch;
  double* H = scratch + (size_t)(M + 1) * NE * NF;
  const double p = alpha + beta, q = gamma;
  double P[3], W[3], PA[3], WP[3], WQ[3], AB[3];
  double ab2 = 0.0, pq2 = 0.0;
  for (int d = 0; d < 3; d++) {
    P[d] = (alpha * A[d] + beta * B[d]) / p;
    AB[d] = A[d] - B[d];
    ab2 += AB[d] * AB[d];
  }
  for (int d = 0; d < 3; d++) {
    W[d] = (p * P[d] + q * Cc[d]) / (p + q);
    PA[d] = P[d] - A[d];
    WP[d] = W[d] - P[d];
    WQ[d] = W[d] - Cc[d];
    pq2 += (P[d] - Cc[d]) * (P[d] - Cc[d]);
  }
  const double rho = p * q / (p + q);
  const double Kab = exp(-alpha * beta / p * ab2);
  const double pref = 2.0 * pow(M_PI, 2.5) / (p * q * sqrt(p + q)) * Kab;
  const double T = rho * pq2;
#define VV(m, e, f) V[((size_t)(m) * NE + (e)) * NF + (f)]
  for (int m = 0; m <= M; m++) VV(m, 0, 0) = pref * oracle_boys(m, T);
  /* build [e|0]^(m) */
  for (int e = 1; e < NE; e++) {
    int E = MX[e] + MY[e] + MZ[e];
    int i = MX[e] > 0 ? 0 : (MY[e] > 0 ? 1 : 2);
    int ex = MX[e] - (i == 0), ey = MY[e] - (i == 1), ez = MZ[e] - (i == 2);
    int e1 = mono_idx(ex, ey, ez);
    int ni = comp(e1, i); /* exponent of e1 in direction i */
    int e2 = -1;
    if (ni > 0) e2 = mono_idx(ex - (i == 0), ey - (i == 1), ez - (i == 2));
    for (int m = 0; m <= M - E; m++) {
      double v = PA[i] * VV(m, e1, 0) + WP[i] * VV(m + 1, e1, 0);
      if (e2 >= 0) v += ni / (2.0 * p) * (VV(m, e2, 0) - rho / p * VV(m + 1, e2, 0));
      VV(m, e, 0) = v;
    }
  }
  /* build [e|f]^(m) */
  for (int f = 1; f < NF; f++) {
    int Fl = MX[f] + MY[f] + MZ[f];
    int i = MX[f] > 0 ? 0 : (MY[f] > 0 ? 1 : 2);
    int fx = MX[f] - (i == 0), fy = MY[f] - (i == 1), fz = MZ[f] - (i == 2);
    int f1 = mono_idx(fx, fy, fz);
    int ni = comp(f1, i);
    int f2 = -1;
    if (ni > 0) f2 = mono_idx(fx - (i == 0), fy - (i == 1), fz - (i == 2));
    for (int e = 0; e < NE; e++) {
      int E = MX[e] + MY[e] + MZ[e];
      int ei = comp(e, i);
      int em = -1;
      if (ei > 0) em = mono_idx(MX[e] - (i == 0), MY[e] - (i == 1), MZ[e] - (i == 2));
      for (int m = 0; m <= M - E - Fl; m++) {
        double v = WQ[i] * VV(m + 1, e, f1); /* (Q-C)_i = 0 for a single ket Gaussian */
        if (f2 >= 0) v += ni / (2.0 * q) * (VV(m, e, f2) - rho / q * VV(m + 1, e, f2));
        if (em >= 0) v += ei / (2.0 * (p + q)) * VV(m + 1, em, f1);
        VV(m, e, f) = v;
      }
    }
  }
  /* horizontal transfer to (a b|c), one ket component at a time */
  const int NB = nm_upto(lb);
  const int na = ncart_l(la), nb = ncart_l(lb), nc = ncart_l(lc);
  const int a0 = nm_upto(la - 1), b0 = nm_upto(lb - 1), c0 = nm_upto(lc - 1);
#define HH(e, b) H[(size_t)(e) * NB + (b)]
  for (int fc = 0; fc < nc; fc++) {
    int f = c0 + fc;
    for (int e = 0; e < NE; e++) HH(e, 0) = VV(0, e, f);
    for (int b = 1; b < NB; b++) {
      int Lb = MX[b] + MY[b] + MZ[b];
      int i = MX[b] > 0 ? 0 : (MY[b] > 0 ? 1 : 2);
      int b1 = mono_idx(MX[b] - (i == 0), MY[b] - (i == 1), MZ[b] - (i == 2));
      for (int e = nm_upto(la - 1); e < nm_upto(Le - Lb); e++) {
        int ep = mono_idx(MX[e] + (i == 0), MY[e] + (i == 1), MZ[e] + (i == 2));
        HH(e, b) = HH(ep, b1) + AB[i] * HH(e, b1);
      }
    }
    for (int ia = 0; ia < na; ia++)
      for (int ib = 0; ib < nb; ib++) out[((size_t)ia * nb + ib) * nc + fc] = HH(a0 + ia, b0 + ib);
  }
#undef HH
#undef VV
}

/* ---------------------------------------------------------------- basis */
typedef struct {
  int n;
  const int* atom;
  const int* l;
  const double* ex;
  int* off; /* first function of each shell */
  int nfun;
} basis_t;

static void basis_init(basis_t* b, int n, const int* atom, const int* l, const double* ex) {
  b->n = n; b->atom = atom; b->l = l; b->ex = ex;
  b->off = (int*)malloc(sizeof(int) * (n + 1));
  int o = 0;
  for (int s = 0; s < n; s++) { b->off[s] = o; o += ncart_l(l[s]); }
  b->off[n] = o;
  b->nfun = o;
}
static void basis_free(basis_t* b) { free(b->off); }

static void shell_norms(int l, double ex, double* nrm) {
  int L = l, k = 0;
  for (int lx = L; lx >= 0; lx--)
    for (int ly = L - lx; ly >= 0; ly--) nrm[k++] = cart_norm(lx, ly, L - lx - ly, ex);
}

int oracle_nfun(int n, const int* l) {
  int o = 0;
  for (int s = 0; s < n; s++) o += ncart_l(l[s]);
  return o;
}

/* (mu nu|P) -> out[nao][nao][naux], both orderings of mu,nu written. */
void oracle_int3c(const double* coords, int nsh, const int* sh_atom, const int* sh_l,
                  const double* sh_ex, int nax, const int* ax_atom, const int* ax_l,
                  const double* ax_ex, double* out) {
  init_tables();
  basis_t bs, ba;
  basis_init(&bs, nsh, sh_atom, sh_l, sh_ex);
  basis_init(&ba, nax, ax_atom, ax_l, ax_ex);
  const int nao = bs.nfun, naux = ba.nfun;
#pragma omp parallel
  {
    double* scr = (double*)malloc(sizeof(double) * scratch_size(4, 4, 3));
    double buf[6 * 6 * 10], na_[10], nb_[10], nc_[10];
#pragma omp for schedule(dynamic)
    for (int sab = 0; sab < nsh * nsh; sab++) {
      int sa = sab / nsh, sb = sab % nsh;
      if (sb < sa) continue;
      shell_norms(sh_l[sa], sh_ex[sa], na_);
      shell_norms(sh_l[sb], sh_ex[sb], nb_);
      int na = ncart_l(sh_l[sa]), nb = ncart_l(sh_l[sb]);
      for (int sc = 0; sc < nax; sc++) {
        shell_norms(ax_l[sc], ax_ex[sc], nc_);
        int nc = ncart_l(ax_l[sc]);
        prim3c(sh_l[sa], sh_l[sb], ax_l[sc], sh_ex[sa], coords + 3 * sh_atom[sa], sh_ex[sb],
               coords + 3 * sh_atom[sb], ax_ex[sc], coords + 3 * ax_atom[sc], buf, scr);
        for (int i = 0; i < na; i++)
          for (int j = 0; j < nb; j++)
            for (int k = 0; k < nc; k++) {
              double v = buf[(i * nb + j) * nc + k] * na_[i] * nb_[j] * nc_[k];
              int mu = bs.off[sa] + i, nu = bs.off[sb] + j, P = ba.off[sc] + k;
              out[((size_t)mu * nao + nu) * naux + P] = v;
              out[((size_t)nu * nao + mu) * naux + P] = v;
            }
      }
    }
    free(scr);
  }
  basis_free(&bs);
  basis_free(&ba);
}

/* (P|Q) -> out[naux][naux] */
void oracle_int2c(const double* coords, int nax, const int* ax_atom, const int* ax_l,
                  const double* ax_ex, double* out) {
  init_tables();
  basis_t ba;
  basis_init(&ba, nax, ax_atom, ax_l, ax_ex);
  const int naux = ba.nfun;
  double* scr = (double*)malloc(sizeof(double) * scratch_size(4, 0, 4));
  double buf[100], np_[10], nq_[10];
  for (int sp = 0; sp < nax; sp++)
    for (int sq = 0; sq < nax; sq++) {
      shell_norms(ax_l[sp], ax_ex[sp], np_);
      shell_norms(ax_l[sq], ax_ex[sq], nq_);
      int n1 = ncart_l(ax_l[sp]), n2 = ncart_l(ax_l[sq]);
      const double* A = coords + 3 * ax_atom[sp];
      prim3c(ax_l[sp], 0, ax_l[sq], ax_ex[sp], A, 0.0, A, ax_ex[sq], coords + 3 * ax_atom[sq],
             buf, scr);
      for (int i = 0; i < n1; i++)
        for (int k = 0; k < n2; k++)
          out[(size_t)(ba.off[sp] + i) * naux + ba.off[sq] + k] = buf[i * n2 + k] * np_[i] * nq_[k];
    }
  free(scr);
  basis_free(&ba);
}

/*
 * Derivatives of one primitive triple with respect to all three centres,
 * each taken directly from the primitive derivative rule:
 * out[centre 0..2][xyz][ia][ib][ic] (raw, unnormalised).
 */
static void prim3c_deriv(int la, int lb, int lc, double alpha, const double* A, double beta,
                         const double* B, double gamma, const double* Cc, int want_a,
                         int want_b, int want_c, double* out, double* scr) {
  const int na = ncart_l(la), nb = ncart_l(lb), nc = ncart_l(lc);
  const int n = na * nb * nc;
  double up[15 * 15 * 10], dn[15 * 15 * 10];
  memset(out, 0, sizeof(double) * 9 * n);
  for (int cen = 0; cen < 3; cen++) {
    if ((cen == 0 && !want_a) || (cen == 1 && !want_b) || (cen == 2 && !want_c)) continue;
    int lu[3] = {la, lb, lc};
    int ld[3] = {la, lb, lc};
    lu[cen] += 1;
    ld[cen] -= 1;
    double ex = cen == 0 ? alpha : (cen == 1 ? beta : gamma);
    prim3c(lu[0], lu[1], lu[2], alpha, A, beta, B, gamma, Cc, up, scr);
    int have_dn = ld[cen] >= 0;
    if (have_dn) prim3c(ld[0], ld[1], ld[2], alpha, A, beta, B, gamma, Cc, dn, scr);
    int nu1 = ncart_l(lu[1]), nu2 = ncart_l(lu[2]);
    int nd1 = have_dn ? ncart_l(ld[1]) : 0, nd2 = have_dn ? ncart_l(ld[2]) : 0;
    int a0 = nm_upto(la - 1), b0 = nm_upto(lb - 1), c0 = nm_upto(lc - 1);
    for (int ia = 0; ia < na; ia++)
      for (int ib = 0; ib < nb; ib++)
        for (int ic = 0; ic < nc; ic++) {
          int mono[3] = {a0 + ia, b0 + ib, c0 + ic};
          for (int d = 0; d < 3; d++) {
            int mu[3], md[3];
            for (int t = 0; t < 3; t++) { mu[t] = mono[t]; md[t] = mono[t]; }
            int cx = MX[mono[cen]], cy = MY[mono[cen]], cz = MZ[mono[cen]];
            int cd = d == 0 ? cx : (d == 1 ? cy : cz);
            mu[cen] = mono_idx(cx + (d == 0), cy + (d == 1), cz + (d == 2));
            int iu0 = mu[0] - nm_upto(lu[0] - 1), iu1 = mu[1] - nm_upto(lu[1] - 1),
                iu2 = mu[2] - nm_upto(lu[2] - 1);
            double v = 2.0 * ex * up[(iu0 * nu1 + iu1) * nu2 + iu2];
            if (cd > 0) {
              md[cen] = mono_idx(cx - (d == 0), cy - (d == 1), cz - (d == 2));
              int id0 = md[0] - nm_upto(ld[0] - 1), id1 = md[1] - nm_upto(ld[1] - 1),
                  id2 = md[2] - nm_upto(ld[2] - 1);
              v -= cd * dn[(id0 * nd1 + id1) * nd2 + id2];
            }
            out[(cen * 3 + d) * n + (ia * nb + ib) * nc + ic] = v;
          }
        }
  }
}

/* Exported for the per-integral pins: normalised derivatives of one shell
 * triple w.r.t. each centre, out[3 centres][3][na][nb][nc]. */
void oracle_int3c_triple_deriv(int la, double alpha, const double* A, int lb, double beta,
                               const double* B, int lc, double gamma, const double* Cc,
                               double* out) {
  init_tables();
  double* scr = (double*)malloc(sizeof(double) * scratch_size(4, 4, 3));
  double na_[10], nb_[10], nc_[10];
  shell_norms(la, alpha, na_);
  shell_norms(lb, beta, nb_);
  shell_norms(lc, gamma, nc_);
  int na = ncart_l(la), nb = ncart_l(lb), nc = ncart_l(lc), n = na * nb * nc;
  prim3c_deriv(la, lb, lc, alpha, A, beta, B, gamma, Cc, 1, 1, 1, out, scr);
  for (int k = 0; k < 9; k++)
    for (int i = 0; i < na; i++)
      for (int j = 0; j < nb; j++)
        for (int c = 0; c < nc; c++) out[k * n + (i * nb + j) * nc + c] *= na_[i] * nb_[j] * nc_[c];
  free(scr);
}

/* Normalised (a b|c) of one shell triple, out[na][nb][nc]. */
void oracle_int3c_triple(int la, double alpha, const double* A, int lb, double beta,
                         const double* B, int lc, double gamma, const double* Cc, double* out) {
  init_tables();
  double* scr = (double*)malloc(sizeof(double) * scratch_size(4, 4, 3));
  double na_[10], nb_[10], nc_[10];
  shell_norms(la, alpha, na_);
  shell_norms(lb, beta, nb_);
  shell_norms(lc, gamma, nc_);
  int na = ncart_l(la), nb = ncart_l(lb), nc = ncart_l(lc);
  prim3c(la, lb, lc, alpha, A, beta, B, gamma, Cc, out, scr);
  for (int i = 0; i < na; i++)
    for (int j = 0; j < nb; j++)
      for (int c = 0; c < nc; c++) out[(i * nb + j) * nc + c] *= na_[i] * nb_[j] * nc_[c];
  free(scr);
}

/*
 * d(mu nu|P)/dR_{atom,x/y/z} -> out[3][nao][nao][naux]: the sum of the
 * derivatives of every centre that sits on `atom`.
 */
void oracle_int3c_deriv_atom(int atom, const double* coords, int nsh, const int* sh_atom,
                             const int* sh_l, const double* sh_ex, int nax, const int* ax_atom,
                             const int* ax_l, const double* ax_ex, double* out) {
  init_tables();
  basis_t bs, ba;
  basis_init(&bs, nsh, sh_atom, sh_l, sh_ex);
  basis_init(&ba, nax, ax_atom, ax_l, ax_ex);
  const int nao = bs.nfun, naux = ba.nfun;
  const size_t plane = (size_t)nao * nao * naux;
  memset(out, 0, sizeof(double) * 3 * plane);
#pragma omp parallel
  {
    double* scr = (double*)malloc(sizeof(double) * scratch_size(4, 4, 3));
    double* d = (double*)malloc(sizeof(double) * 9 * 6 * 6 * 6);  /* AO and aux shells up to d */
    double na_[10], nb_[10], nc_[10];
#pragma omp for schedule(dynamic)
    for (int sab = 0; sab < nsh * nsh; sab++) {
      int sa = sab / nsh, sb = sab % nsh;
      if (sb < sa) continue;
      shell_norms(sh_l[sa], sh_ex[sa], na_);
      shell_norms(sh_l[sb], sh_ex[sb], nb_);
      int na = ncart_l(sh_l[sa]), nb = ncart_l(sh_l[sb]);
      for (int sc = 0; sc < nax; sc++) {
        int wa = sh_atom[sa] == atom, wb = sh_atom[sb] == atom, wc = ax_atom[sc] == atom;
        if (!(wa || wb || wc)) continue;
        shell_norms(ax_l[sc], ax_ex[sc], nc_);
        int nc = ncart_l(ax_l[sc]), n = na * nb * nc;
        prim3c_deriv(sh_l[sa], sh_l[sb], ax_l[sc], sh_ex[sa], coords + 3 * sh_atom[sa],
                     sh_ex[sb], coords + 3 * sh_atom[sb], ax_ex[sc], coords + 3 * ax_atom[sc],
                     wa, wb, wc, d, scr);
        for (int x = 0; x < 3; x++)
          for (int i = 0; i < na; i++)
            for (int j = 0; j < nb; j++)
              for (int k = 0; k < nc; k++) {
                int o = (i * nb + j) * nc + k;
                double v = (d[(0 * 3 + x) * n + o] + d[(1 * 3 + x) * n + o] +
                            d[(2 * 3 + x) * n + o]) *
                           na_[i] * nb_[j] * nc_[k];
                int mu = bs.off[sa] + i, nu = bs.off[sb] + j, P = ba.off[sc] + k;
                out[x * plane + ((size_t)mu * nao + nu) * naux + P] = v;
                out[x * plane + ((size_t)nu * nao + mu) * naux + P] = v;
              }
      }
    }
    free(d);
    free(scr);
  }
  basis_free(&bs);
  basis_free(&ba);
}

/* d(P|Q)/dR_{atom,x/y/z} -> out[3][naux][naux] */
void oracle_int2c_deriv_atom(int atom, const double* coords, int nax, const int* ax_atom,
                             const int* ax_l, const double* ax_ex, double* out) {
  init_tables();
  basis_t ba;
  basis_init(&ba, nax, ax_atom, ax_l, ax_ex);
  const int naux = ba.nfun;
  memset(out, 0, sizeof(double) * 3 * naux * naux);
  double* scr = (double*)malloc(sizeof(double) * scratch_size(4, 4, 4));
  double d[9 * 100], np_[10], nq_[10];
  for (int sp = 0; sp < nax; sp++)
    for (int sq = 0; sq < nax; sq++) {
      int wp = ax_atom[sp] == atom, wq = ax_atom[sq] == atom;
      if (!(wp || wq)) continue;
      shell_norms(ax_l[sp], ax_ex[sp], np_);
      shell_norms(ax_l[sq], ax_ex[sq], nq_);
      int n1 = ncart_l(ax_l[sp]), n2 = ncart_l(ax_l[sq]), n = n1 * n2;
      const double* A = coords + 3 * ax_atom[sp];
      /* (p 1|q): the middle "function" is the constant 1 (exponent 0) at A;
         it carries no coordinate dependence, so only centres 0 and 2 move. */
      prim3c_deriv(ax_l[sp], 0, ax_l[sq], ax_ex[sp], A, 0.0, A, ax_ex[sq],
                   coords + 3 * ax_atom[sq], wp, 0, wq, d, scr);
      for (int x = 0; x < 3; x++)
        for (int i = 0; i < n1; i++)
          for (int k = 0; k < n2; k++) {
            int o = i * n2 + k;
            out[(size_t)x * naux * naux + (size_t)(ba.off[sp] + i) * naux + ba.off[sq] + k] =
                (d[(0 * 3 + x) * n + o] + d[(2 * 3 + x) * n + o]) * np_[i] * nq_[k];
          }
    }
  free(scr);
  basis_free(&ba);
}

/* AO overlap by the Obara-Saika one-electron recurrence, out[nao][nao]. */
static double os_overlap_1d(int i, int j, double a, double b, double A, double B) {
  double p = a + b, P = (a * A + b * B) / p;
  double PA = P - A, PB = P - B;
  double s[12][12];
  s[0][0] = sqrt(M_PI / p) * exp(-a * b / p * (A - B) * (A - B));
  for (int u = 0; u <= i; u++)
    for (int v = 0; v <= j; v++) {
      if (u == 0 && v == 0) continue;
      double r;
      if (u > 0) {
        r = PA * s[u - 1][v];
        if (u > 1) r += (u - 1) / (2 * p) * s[u - 2][v];
        if (v > 0) r += v / (2 * p) * s[u - 1][v - 1];
      } else {
        r = PB * s[u][v - 1];
        if (v > 1) r += (v - 1) / (2 * p) * s[u][v - 2];
      }
      s[u][v] = r;
    }
  return s[i][j];
}

void oracle_overlap(const double* coords, int nsh, const int* sh_atom, const int* sh_l,
                    const double* sh_ex, double* out) {
  init_tables();
  basis_t bs;
  basis_init(&bs, nsh, sh_atom, sh_l, sh_ex);
  const int nao = bs.nfun;
  for (int sa = 0; sa < nsh; sa++)
    for (int sb = 0; sb < nsh; sb++) {
      const double* A = coords + 3 * sh_atom[sa];
      const double* B = coords + 3 * sh_atom[sb];
      int la = sh_l[sa], lb = sh_l[sb];
      int a0 = nm_upto(la - 1), b0 = nm_upto(lb - 1);
      for (int i = 0; i < ncart_l(la); i++)
        for (int j = 0; j < ncart_l(lb); j++) {
          int ka = a0 + i, kb = b0 + j;
          double v = cart_norm(MX[ka], MY[ka], MZ[ka], sh_ex[sa]) *
                     cart_norm(MX[kb], MY[kb], MZ[kb], sh_ex[sb]);
          v *= os_overlap_1d(MX[ka], MX[kb], sh_ex[sa], sh_ex[sb], A[0], B[0]);
          v *= os_overlap_1d(MY[ka], MY[kb], sh_ex[sa], sh_ex[sb], A[1], B[1]);
          v *= os_overlap_1d(MZ[ka], MZ[kb], sh_ex[sa], sh_ex[sb], A[2], B[2]);
          out[(size_t)(bs.off[sa] + i) * nao + bs.off[sb] + j] = v;
        }
    }
  basis_free(&bs);
}
