// Integral engine for the ris auxiliary basis (Sec. 2.2): three-centre
// (mu nu|P) and two-centre (P|Q) Coulomb integrals and their first nuclear
// derivatives, as used by Eq. (g_modified) and by the RI derivative formula
// that closes Sec. 2.2.
//
// Method: McMurchie-Davidson.  The bra Gaussian product is expanded in
// Hermite Gaussians with coefficients E^{ij}_t (one set per cartesian
// direction); the Coulomb interaction with the auxiliary Gaussian reduces to
// the Hermite integrals R_tuv(rho, P-C), built from the Boys function
// F_n(T) by the standard downward-in-n recursion.  A p auxiliary function
// (x-C_x)e^{-g r_C^2} = (1/2g) d/dC_x e^{-g r_C^2} enters as -1/(2g) R_{t+1}.
// Derivatives use d/dA_x x_A^i e^{-a x_A^2} = 2a x_A^{i+1}.. - i x_A^{i-1}..,
// i.e. E coefficients with i +- 1; the auxiliary-centre derivative follows
// from translational invariance where it is needed.
//
// Boys function: F_m(T) for T < 40 by an 8-term Taylor expansion about the
// nearest point of a table spaced 0.05 (truncation < 4e-18 relative) and
// downward recursion F_m = (2T F_{m+1} + e^{-T})/(2m+1); for T >= 40 by
// F_0 = sqrt(pi/T)/2 (erf(sqrt T) = 1 to 1e-18) and upward recursion.  The
// table is filled on the host by composite Gauss-Legendre quadrature of the
// definition F_m(T) = int_0^1 t^{2m} e^{-T t^2} dt.
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "ints.cuh"

namespace ris {

// ------------------------------------------------------------------ Boys
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; i++) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; it++) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; k++) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; k++) {
      double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

static std::vector<double> make_boys_table() {
  // composite 32-point Gauss-Legendre on 32 panels of [0,1]; the integrand
  // t^{2m} e^{-T t^2} is evaluated once per node for all m; Kahan summation.
  std::vector<double> gx, gw;
  gauss_legendre(32, gx, gw);
  const int panels = 32, nq = 32 * panels;
  std::vector<double> tq(nq), wq(nq), ex(nq);
  for (int pnl = 0; pnl < panels; pnl++) {
    const double a = (double)pnl / panels, b = (double)(pnl + 1) / panels;
    for (int i = 0; i < 32; i++) {
      tq[pnl * 32 + i] = 0.5 * (b - a) * gx[i] + 0.5 * (a + b);
      wq[pnl * 32 + i] = 0.5 * (b - a) * gw[i];
    }
  }
  std::vector<double> tab((size_t)kBoysNT * (kBoysM + 1));
  for (int k = 0; k < kBoysNT; k++) {
    const double T = k * kBoysDT;
    for (int q = 0; q < nq; q++) ex[q] = wq[q] * exp(-T * tq[q] * tq[q]);
    for (int m = 0; m <= kBoysM; m++) {
      double s = 0.0, comp = 0.0;
      for (int q = 0; q < nq; q++) {
        const double y = ex[q] - comp;
        const double t = s + y;
        comp = (t - s) - y;
        s = t;
        ex[q] *= tq[q] * tq[q];  // next m
      }
      tab[(size_t)k * (kBoysM + 1) + m] = s;
    }
  }
  return tab;
}

const double* boys_table_device(int device) {
  static std::mutex mu;
  static std::map<int, double*> per_dev;
  static std::vector<double> host;
  std::lock_guard<std::mutex> g(mu);
  auto it = per_dev.find(device);
  if (it != per_dev.end()) return it->second;
  if (host.empty()) host = make_boys_table();
  double* d = nullptr;
  RIS_ALLOC(cudaMalloc(&d, host.size() * sizeof(double)));
  RIS_CUDA(cudaMemcpy(d, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice));
  per_dev[device] = d;
  return d;
}

template <int M>
__device__ __forceinline__ void boys(double T, const double* __restrict__ tab, double (&F)[M + 1]) {
  if (T < kBoysTmax) {
    int k = __double2int_rn(T * (1.0 / kBoysDT));
    double dt = T - k * kBoysDT;
    const double* row = tab + k * (kBoysM + 1) + M;
    double f = __ldg(row + kBoysTaylor - 1);
#pragma unroll
    for (int j = kBoysTaylor - 1; j >= 1; j--) f = __ldg(row + j - 1) - dt * f * (1.0 / j);
    F[M] = f;
    double e = exp(-T);
#pragma unroll
    for (int m = M - 1; m >= 0; m--) F[m] = (2.0 * T * F[m + 1] + e) * (1.0 / (2 * m + 1));
  } else {
    double e = exp(-T);
    double inv2T = 0.5 / T;
    F[0] = 0.5 * sqrt(M_PI / T);
#pragma unroll
    for (int m = 0; m < M; m++) F[m + 1] = ((2 * m + 1) * F[m] - e) * inv2T;
  }
}

// Boys values for a batch of (m, T), used by the parity tests.
__global__ void k_boys_probe(int n, const int* m, const double* T, const double* tab, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double f[10];
  boys<9>(T[i], tab, f);
  out[i] = f[m[i]];
}

// ------------------------------------------------------------------ Hermite machinery
__host__ __device__ constexpr int hidx(int t, int u, int v) {
  return (t + u + v) * (t + u + v + 1) * (t + u + v + 2) / 6 +
         (u + v) * (u + v + 1) / 2 + v;
}
template <int L>
struct NH {
  static constexpr int n = (L + 1) * (L + 2) * (L + 3) / 6;
};

// E[d][i][j][t] for i <= IA, j <= JB.
template <int IA, int JB>
__device__ __forceinline__ void hermite_E(double p, const double (&PA)[3], const double (&PB)[3],
                                          double (&E)[3][IA + 1][JB + 1][IA + JB + 1]) {
  const double o2p = 0.5 / p;
#pragma unroll
  for (int d = 0; d < 3; d++) {
#pragma unroll
    for (int i = 0; i <= IA; i++)
#pragma unroll
      for (int j = 0; j <= JB; j++)
#pragma unroll
        for (int t = 0; t <= IA + JB; t++) E[d][i][j][t] = 0.0;
    E[d][0][0][0] = 1.0;
#pragma unroll
    for (int i = 1; i <= IA; i++)
#pragma unroll
      for (int t = 0; t <= i; t++) {
        double v = PA[d] * E[d][i - 1][0][t];
        if (t > 0) v += o2p * E[d][i - 1][0][t - 1];
        if (t + 1 <= i - 1) v += (t + 1) * E[d][i - 1][0][t + 1];
        E[d][i][0][t] = v;
      }
#pragma unroll
    for (int j = 1; j <= JB; j++)
#pragma unroll
      for (int i = 0; i <= IA; i++)
#pragma unroll
        for (int t = 0; t <= i + j; t++) {
          double v = PB[d] * E[d][i][j - 1][t];
          if (t > 0) v += o2p * E[d][i][j - 1][t - 1];
          if (t + 1 <= i + j - 1) v += (t + 1) * E[d][i][j - 1][t + 1];
          E[d][i][j][t] = v;
        }
  }
}

// R[hidx(t,u,v)] = R^{(0)}_{tuv}(rho, X,Y,Z) for t+u+v <= L, built in place
// from n = L down to 0.
template <int L>
__device__ __forceinline__ void hermite_R(double rho, double X, double Y, double Z,
                                          const double (&F)[L + 1], double (&R)[NH<L>::n]) {
  double pw[L + 1];
  pw[0] = 1.0;
#pragma unroll
  for (int n = 1; n <= L; n++) pw[n] = pw[n - 1] * (-2.0 * rho);
  R[0] = pw[L] * F[L];
#pragma unroll
  for (int n = L - 1; n >= 0; n--) {
#pragma unroll
    for (int N = L - n; N >= 1; N--) {
#pragma unroll
      for (int t = N; t >= 0; t--) {
#pragma unroll
        for (int u = N - t; u >= 0; u--) {
          const int v = N - t - u;
          double r;
          if (t > 0) {
            r = X * R[hidx(t - 1, u, v)];
            if (t > 1) r += (t - 1) * R[hidx(t - 2, u, v)];
          } else if (u > 0) {
            r = Y * R[hidx(t, u - 1, v)];
            if (u > 1) r += (u - 1) * R[hidx(t, u - 2, v)];
          } else {
            r = Z * R[hidx(t, u, v - 1)];
            if (v > 1) r += (v - 1) * R[hidx(t, u, v - 2)];
          }
          R[hidx(t, u, v)] = r;
        }
      }
    }
    R[0] = pw[n] * F[n];
  }
}

// cartesian component c of shell l: exponents
__host__ __device__ constexpr int cx_(int l, int c) {
  return l == 0 ? 0 : (l == 1 ? (c == 0 ? 1 : 0) : (c == 0 ? 2 : (c == 1 || c == 2) ? 1 : 0));
}
__host__ __device__ constexpr int cy_(int l, int c) {
  return l == 0 ? 0 : (l == 1 ? (c == 1 ? 1 : 0) : (c == 1 || c == 4) ? 1 : (c == 3 ? 2 : 0));
}
__host__ __device__ constexpr int cz_(int l, int c) {
  return l - cx_(l, c) - cy_(l, c);
}
// 1/sqrt((2lx-1)!!(2ly-1)!!(2lz-1)!!) for the normalisation of component c
__host__ __device__ constexpr double cfac(int l, int c) {
  return (l == 2 && (c == 0 || c == 3 || c == 5)) ? 0.57735026918962576451 : 1.0;
}

// Hermite expansion of one Cartesian factor x^k exp(-g x^2) of a Gaussian in
// Hermite Gaussians Lambda_tau = (d/dC_x)^tau exp(-g (x - C_x)^2):
//   x^0 = Lambda_0, x^1 = Lambda_1 / (2g), x^2 = Lambda_0 / (2g) + Lambda_2 / (4g^2);
// sgn = -1 applies the ket sign (-1)^tau of the McMurchie-Davidson formula.
__device__ __forceinline__ int herm1(int k, double g, double sgn, int* tau, double* c) {
  if (k <= 1) {  // one term: the s and p auxiliary shells
    tau[0] = k;
    c[0] = k == 0 ? 1.0 : sgn * 0.5 / g;
    return 1;
  }
  tau[0] = 0;  // k == 2
  c[0] = 0.5 / g;
  tau[1] = 2;
  c[1] = 0.25 / (g * g);
  return 2;
}

struct PairGeom {
  double p, PA[3], PB[3], P[3], pref_ab;  // pref_ab = K_ab * nbase_a * nbase_b
};

__device__ __forceinline__ void pair_geom(double a, const double* A, double b, const double* B,
                                          double na, double nb, PairGeom& g) {
  g.p = a + b;
  double ab2 = 0.0;
#pragma unroll
  for (int d = 0; d < 3; d++) {
    g.P[d] = (a * A[d] + b * B[d]) / g.p;
    g.PA[d] = g.P[d] - A[d];
    g.PB[d] = g.P[d] - B[d];
    ab2 += (A[d] - B[d]) * (A[d] - B[d]);
  }
  g.pref_ab = exp(-a * b / g.p * ab2) * na * nb;
}

// ------------------------------------------------------------------ three-centre
template <int LA, int LB, int LC>
__global__ void __launch_bounds__(128) k_int3c(const int* __restrict__ pa, const int* __restrict__ pb,
                                               int p0, int np, const int* __restrict__ auxl,
                                               int nax, const int* __restrict__ sh_atom,
                                               const int* __restrict__ sh_off,
                                               const double* __restrict__ sh_ex,
                                               const double* __restrict__ sh_nb,
                                               const int* __restrict__ ax_atom,
                                               const double* __restrict__ ax_ex,
                                               const double* __restrict__ ax_nb,
                                               const int* __restrict__ ax_jmap,
                                               const int* __restrict__ ax_kmap,
                                               const double* __restrict__ xyz,
                                               const double* __restrict__ boys_tab, int nao,
                                               int nJ, int nK, double* __restrict__ TJ,
                                               double* __restrict__ TK,
                                               const long long* __restrict__ poff,
                                               const int* __restrict__ ax_off) {
  constexpr int L = LA + LB + LC;
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (long long)np * nax) return;
  const int ip = p0 + (int)(tid / nax);
  const int sc = auxl[(int)(tid % nax)];
  const int sa = pa[ip], sb = pb[ip];
  const double* A = xyz + 3 * sh_atom[sa];
  const double* B = xyz + 3 * sh_atom[sb];
  const double* Cc = xyz + 3 * ax_atom[sc];
  PairGeom g;
  pair_geom(sh_ex[sa], A, sh_ex[sb], B, sh_nb[sa], sh_nb[sb], g);
  const double gam = ax_ex[sc];
  const double rho = g.p * gam / (g.p + gam);
  const double X = g.P[0] - Cc[0], Y = g.P[1] - Cc[1], Z = g.P[2] - Cc[2];
  double F[L + 1];
  boys<L>(rho * (X * X + Y * Y + Z * Z), boys_tab, F);
  double R[NH<L>::n];
  hermite_R<L>(rho, X, Y, Z, F, R);
  double E[3][LA + 1][LB + 1][LA + LB + 1];
  hermite_E<LA, LB>(g.p, g.PA, g.PB, E);
  const double pref = 2.0 * 17.493418327624862 /* pi^2.5 */ / (g.p * gam * sqrt(g.p + gam)) *
                      g.pref_ab * ax_nb[sc];
  const int oa = sh_off[sa], ob = sh_off[sb];
  const int jm = ax_jmap[sc], km = ax_kmap[sc];
#pragma unroll 1
  for (int ia = 0; ia < (LA + 1) * (LA + 2) / 2; ia++) {
    const int ax = cx_(LA, ia), ay = cy_(LA, ia), az = cz_(LA, ia);
#pragma unroll 1
    for (int ib = 0; ib < (LB + 1) * (LB + 2) / 2; ib++) {
      const int bx = cx_(LB, ib), by = cy_(LB, ib), bz = cz_(LB, ib);
      const double nab = pref * cfac(LA, ia) * cfac(LB, ib);
#pragma unroll 1
      for (int ic = 0; ic < (LC + 1) * (LC + 2) / 2; ic++) {
        int tx[2], ty[2], tz[2];
        double fx[2], fy[2], fz[2];
        const int nx = herm1(cx_(LC, ic), gam, -1.0, tx, fx);
        const int ny = herm1(cy_(LC, ic), gam, -1.0, ty, fy);
        const int nz = herm1(cz_(LC, ic), gam, -1.0, tz, fz);
        double s = 0.0;
        const int mx = LC <= 1 ? 1 : nx, my = LC <= 1 ? 1 : ny, mz = LC <= 1 ? 1 : nz;
        for (int jx = 0; jx < mx; jx++)
          for (int jy = 0; jy < my; jy++)
            for (int jz = 0; jz < mz; jz++) {
              const int kx = tx[jx], ky = ty[jy], kz = tz[jz];
              double sub = 0.0;
#pragma unroll 1
              for (int t = 0; t <= ax + bx; t++) {
                const double et = E[0][ax][bx][t];
#pragma unroll 1
                for (int u = 0; u <= ay + by; u++) {
                  const double eu = et * E[1][ay][by][u];
#pragma unroll 1
                  for (int v = 0; v <= az + bz; v++)
                    sub += eu * E[2][az][bz][v] * R[hidx(t + kx, u + ky, v + kz)];
                }
              }
              s += fx[jx] * fy[jy] * fz[jz] * sub;
            }
        s *= nab * cfac(LC, ic);
        if (poff) {  // screened-pair storage: one row per function pair of this shell pair
          constexpr int NB = (LB + 1) * (LB + 2) / 2;
          TJ[(size_t)(poff[ip] + ia * NB + ib) * nJ + ax_off[sc] + ic] = s;
          continue;
        }
        const int mu = oa + ia, nu = ob + ib;
        if (jm >= 0) {
          TJ[((size_t)mu * nao + nu) * nJ + jm + ic] = s;
          TJ[((size_t)nu * nao + mu) * nJ + jm + ic] = s;
        }
        if (km >= 0) {
          TK[((size_t)mu * nao + nu) * nK + km + ic] = s;
          TK[((size_t)nu * nao + mu) * nK + km + ic] = s;
        }
      }
    }
  }
}

// d(mu nu|P)/dA_x (A = centre of mu) and d(mu nu|P)/dB_x, written as
// D[x][mu][nu][P] and D[x][nu][mu][P] (computed in FP64, stored as T).
template <int LA, int LB, int LC, class T>
__global__ void __launch_bounds__(128) k_int3c_deriv(
    const int* __restrict__ pa, const int* __restrict__ pb, int p0, int np,
    const int* __restrict__ auxl, int nax, const int* __restrict__ sh_atom,
    const int* __restrict__ sh_off, const double* __restrict__ sh_ex,
    const double* __restrict__ sh_nb, const int* __restrict__ ax_atom,
    const int* __restrict__ ax_off, const double* __restrict__ ax_ex,
    const double* __restrict__ ax_nb, const double* __restrict__ xyz,
    const double* __restrict__ boys_tab, int nao, int naux, T* __restrict__ D) {
  constexpr int L = LA + LB + LC + 1;
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (long long)np * nax) return;
  const int ip = p0 + (int)(tid / nax);
  const int sc = auxl[(int)(tid % nax)];
  const int sa = pa[ip], sb = pb[ip];
  const double* A = xyz + 3 * sh_atom[sa];
  const double* B = xyz + 3 * sh_atom[sb];
  const double* Cc = xyz + 3 * ax_atom[sc];
  PairGeom g;
  const double alpha = sh_ex[sa], beta = sh_ex[sb];
  pair_geom(alpha, A, beta, B, sh_nb[sa], sh_nb[sb], g);
  const double gam = ax_ex[sc];
  const double rho = g.p * gam / (g.p + gam);
  const double X = g.P[0] - Cc[0], Y = g.P[1] - Cc[1], Z = g.P[2] - Cc[2];
  double F[L + 1];
  boys<L>(rho * (X * X + Y * Y + Z * Z), boys_tab, F);
  double R[NH<L>::n];
  hermite_R<L>(rho, X, Y, Z, F, R);
  double E[3][LA + 2][LB + 2][LA + LB + 3];
  hermite_E<LA + 1, LB + 1>(g.p, g.PA, g.PB, E);
  const double pref = 2.0 * 17.493418327624862 / (g.p * gam * sqrt(g.p + gam)) * g.pref_ab *
                      ax_nb[sc];
  const int oa = sh_off[sa], ob = sh_off[sb], oc = ax_off[sc];
  const size_t plane = (size_t)nao * nao * naux;
#pragma unroll 1
  for (int ia = 0; ia < (LA + 1) * (LA + 2) / 2; ia++) {
    const int a_[3] = {cx_(LA, ia), cy_(LA, ia), cz_(LA, ia)};
#pragma unroll 1
    for (int ib = 0; ib < (LB + 1) * (LB + 2) / 2; ib++) {
      const int b_[3] = {cx_(LB, ib), cy_(LB, ib), cz_(LB, ib)};
      const double nab = pref * cfac(LA, ia) * cfac(LB, ib);
#pragma unroll 1
      for (int ic = 0; ic < (LC + 1) * (LC + 2) / 2; ic++) {
        int th[3][2];
        double fh[3][2];
        const int nh[3] = {herm1(cx_(LC, ic), gam, -1.0, th[0], fh[0]),
                           herm1(cy_(LC, ic), gam, -1.0, th[1], fh[1]),
                           herm1(cz_(LC, ic), gam, -1.0, th[2], fh[2])};
        const double sc_ = cfac(LC, ic) * nab;
        const int mu = oa + ia, nu = ob + ib, P = oc + ic;
#pragma unroll 1
        for (int x = 0; x < 3; x++) {
          // differentiated direction x: E -> 2 alpha E^{a+1} - a_x E^{a-1}
          // (centre A) and 2 beta E^{b+1} - b_x E^{b-1} (centre B)
          const int y = (x + 1) % 3, z = (x + 2) % 3;
          const int tx_max = a_[x] + b_[x] + 1;
          double sA = 0.0, sB = 0.0;
#pragma unroll 1
          for (int t = 0; t <= tx_max; t++) {
            const double up = E[x][a_[x] + 1][b_[x]][t];
            const double dn = a_[x] > 0 ? E[x][a_[x] - 1][b_[x]][t] : 0.0;
            const double upb = E[x][a_[x]][b_[x] + 1][t];
            const double dnb = b_[x] > 0 ? E[x][a_[x]][b_[x] - 1][t] : 0.0;
            const double eA = 2.0 * alpha * up - a_[x] * dn;
            const double eB = 2.0 * beta * upb - b_[x] * dnb;
            double r = 0.0;
            // LC <= 1: one Hermite term per axis (loops of length 1 at compile time)
            const int mx = LC <= 1 ? 1 : nh[x], my = LC <= 1 ? 1 : nh[y], mz = LC <= 1 ? 1 : nh[z];
            for (int jx = 0; jx < mx; jx++)
              for (int jy = 0; jy < my; jy++)
                for (int jz = 0; jz < mz; jz++) {
                  const double fc = fh[x][jx] * fh[y][jy] * fh[z][jz];
                  double rr = 0.0;
#pragma unroll 1
                  for (int u = 0; u <= a_[y] + b_[y]; u++) {
                    const double eu = E[y][a_[y]][b_[y]][u];
#pragma unroll 1
                    for (int v = 0; v <= a_[z] + b_[z]; v++) {
                      int tuv[3];
                      tuv[x] = t + th[x][jx];
                      tuv[y] = u + th[y][jy];
                      tuv[z] = v + th[z][jz];
                      rr += eu * E[z][a_[z]][b_[z]][v] * R[hidx(tuv[0], tuv[1], tuv[2])];
                    }
                  }
                  r += fc * rr;
                }
            sA += eA * r;
            sB += eB * r;
          }
          D[x * plane + ((size_t)mu * nao + nu) * naux + P] = (T)(sA * sc_);
          D[x * plane + ((size_t)nu * nao + mu) * naux + P] = (T)(sB * sc_);
        }
      }
    }
  }
}

// ------------------------------------------------------------------ two-centre
// (P|Q) and d(P|Q)/dP_x, l <= 1 on both sides.
__global__ void k_int2c(int nsh, const int* __restrict__ atom, const int* __restrict__ lq,
                        const int* __restrict__ off, const double* __restrict__ ex,
                        const double* __restrict__ nbase, const double* __restrict__ xyz,
                        const double* __restrict__ boys_tab, int naux, double* __restrict__ M,
                        double* __restrict__ dM) {
  int tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= nsh * nsh) return;
  const int sp = tid / nsh, sq = tid % nsh;
  const double a = ex[sp], c = ex[sq];
  const double* A = xyz + 3 * atom[sp];
  const double* Cc = xyz + 3 * atom[sq];
  const double rho = a * c / (a + c);
  const double X = A[0] - Cc[0], Y = A[1] - Cc[1], Z = A[2] - Cc[2];
  constexpr int LM = 2 * kMaxLAux + 1;  // (P|Q) and its first derivative
  double F[LM + 1];
  boys<LM>(rho * (X * X + Y * Y + Z * Z), boys_tab, F);
  double R[NH<LM>::n];
  hermite_R<LM>(rho, X, Y, Z, F, R);
  const double pref = 2.0 * 17.493418327624862 / (a * c * sqrt(a + c)) * nbase[sp] * nbase[sq];
  const int l1 = lq[sp], l2 = lq[sq];
  for (int i = 0; i < ncart(l1); i++) {
    int t1[3][2], n1[3];
    double f1[3][2];
    n1[0] = herm1(cx_(l1, i), a, 1.0, t1[0], f1[0]);
    n1[1] = herm1(cy_(l1, i), a, 1.0, t1[1], f1[1]);
    n1[2] = herm1(cz_(l1, i), a, 1.0, t1[2], f1[2]);
    for (int k = 0; k < ncart(l2); k++) {
      int t2[3][2], n2[3];
      double f2[3][2];
      n2[0] = herm1(cx_(l2, k), c, -1.0, t2[0], f2[0]);
      n2[1] = herm1(cy_(l2, k), c, -1.0, t2[1], f2[1]);
      n2[2] = herm1(cz_(l2, k), c, -1.0, t2[2], f2[2]);
      double m = 0.0, d0 = 0.0, d1 = 0.0, d2 = 0.0;
      for (int ax = 0; ax < n1[0]; ax++)
        for (int ay = 0; ay < n1[1]; ay++)
          for (int az = 0; az < n1[2]; az++)
            for (int bx = 0; bx < n2[0]; bx++)
              for (int by = 0; by < n2[1]; by++)
                for (int bz = 0; bz < n2[2]; bz++) {
                  const double f = f1[0][ax] * f1[1][ay] * f1[2][az] * f2[0][bx] * f2[1][by] *
                                   f2[2][bz];
                  const int t = t1[0][ax] + t2[0][bx], u = t1[1][ay] + t2[1][by],
                            v = t1[2][az] + t2[2][bz];
                  m += f * R[hidx(t, u, v)];
                  // d/dA_x R_tuv(A - C) = R_{t+1,u,v}
                  d0 += f * R[hidx(t + 1, u, v)];
                  d1 += f * R[hidx(t, u + 1, v)];
                  d2 += f * R[hidx(t, u, v + 1)];
                }
      const double nf = pref * cfac(l1, i) * cfac(l2, k);
      const size_t o = (size_t)(off[sp] + i) * naux + off[sq] + k;
      M[o] = nf * m;
      dM[o] = nf * d0;
      dM[(size_t)naux * naux + o] = nf * d1;
      dM[(size_t)2 * naux * naux + o] = nf * d2;
    }
  }
}

// ------------------------------------------------------------------ pairs
// Screening estimate of max |(mu nu|P)| over the pair: the L1 norm bound of
// the Gaussian product, N_a N_b K_ab (pi/p)^{3/2} (1+|PA|+p^-1/2)^la
// (1+|PB|+p^-1/2)^lb, times the largest auxiliary potential (folded into thr).
__device__ __forceinline__ double pair_bound(double a, const double* A, int la, double na, double b,
                                             const double* B, int lb, double nb) {
  const double p = a + b;
  double ab2 = 0.0, pa2 = 0.0, pb2 = 0.0;
  for (int d = 0; d < 3; d++) {
    double P = (a * A[d] + b * B[d]) / p;
    ab2 += (A[d] - B[d]) * (A[d] - B[d]);
    pa2 += (P - A[d]) * (P - A[d]);
    pb2 += (P - B[d]) * (P - B[d]);
  }
  const double s = 1.0 / sqrt(p);
  double v = na * nb * exp(-a * b / p * ab2) * pow(M_PI / p, 1.5);
  for (int k = 0; k < la; k++) v *= 1.0 + sqrt(pa2) + s;
  for (int k = 0; k < lb; k++) v *= 1.0 + sqrt(pb2) + s;
  return v;
}

constexpr int kPairBlock = 256;

__device__ __forceinline__ int pair_key(int tid, int nsh, const int* l, const int* atom,
                                        const double* ex, const double* nb, const double* xyz,
                                        double thr, int& s1, int& s2) {
  const int a = tid / nsh, b = tid % nsh;
  if (b < a) return 7;
  if (l[a] >= l[b]) {
    s1 = a;
    s2 = b;
  } else {
    s1 = b;
    s2 = a;
  }
  const double bound = pair_bound(ex[s1], xyz + 3 * atom[s1], l[s1], nb[s1], ex[s2],
                                  xyz + 3 * atom[s2], l[s2], nb[s2]);
  if (!(bound >= thr)) return 7;
  return l[s1] * (l[s1] + 1) / 2 + l[s2];
}

__global__ void k_pair_count(int nsh, const int* l, const int* atom, const double* ex,
                             const double* nb, const double* xyz, double thr, int* counts) {
  __shared__ int c[8];
  if (threadIdx.x < 8) c[threadIdx.x] = 0;
  __syncthreads();
  const int tid = blockIdx.x * kPairBlock + threadIdx.x;
  if (tid < nsh * nsh) {
    int s1, s2;
    int k = pair_key(tid, nsh, l, atom, ex, nb, xyz, thr, s1, s2);
    atomicAdd(&c[k], 1);
  }
  __syncthreads();
  if (threadIdx.x < 8) counts[blockIdx.x * 8 + threadIdx.x] = c[threadIdx.x];
}

// Exclusive offsets, key-major then block order; totals[8] = class sizes.
__global__ void k_pair_scan(int nblk, const int* counts, int* offs, int* totals) {
  __shared__ int tot[8];
  const int k = threadIdx.x;
  if (k < 8) {
    int s = 0;
    for (int b = 0; b < nblk; b++) s += counts[b * 8 + k];
    tot[k] = s;
  }
  __syncthreads();
  if (k < 8) {
    int base = 0;
    for (int j = 0; j < k; j++) base += tot[j];
    for (int b = 0; b < nblk; b++) {
      offs[b * 8 + k] = base;
      base += counts[b * 8 + k];
    }
    totals[k] = tot[k];
  }
}

__global__ void k_pair_scatter(int nsh, const int* l, const int* atom, const double* ex,
                               const double* nb, const double* xyz, double thr, const int* offs,
                               int* out_a, int* out_b) {
  __shared__ int warp_cnt[kPairBlock / 32][8];
  const int tid = blockIdx.x * kPairBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int s1 = 0, s2 = 0, k = 7;
  if (tid < nsh * nsh) k = pair_key(tid, nsh, l, atom, ex, nb, xyz, thr, s1, s2);
  int rank = 0;
  for (int key = 0; key < 8; key++) {
    unsigned m = __ballot_sync(0xffffffffu, k == key);
    if (k == key) rank = __popc(m & ((1u << lane) - 1u));
    if (lane == 0) warp_cnt[w][key] = __popc(m);
  }
  __syncthreads();
  if (k < 7) {
    int o = offs[blockIdx.x * 8 + k] + rank;
    for (int j = 0; j < w; j++) o += warp_cnt[j][k];
    out_a[o] = s1;
    out_b[o] = s2;
  }
}

void build_pairs(const ShellSet& ao, const double* d_coords, double thr, PairList& pl,
                 void* /*scratch*/, cudaStream_t st) {
  free_pairs(pl, st);
  const int nsh = ao.n;
  const int nitem = nsh * nsh;
  const int nblk = cdiv(nitem, kPairBlock);
  int *counts = nullptr, *offs = nullptr, *totals = nullptr;
  RIS_ALLOC(cudaMallocAsync(&counts, sizeof(int) * 8 * nblk, st));
  RIS_ALLOC(cudaMallocAsync(&offs, sizeof(int) * 8 * nblk, st));
  RIS_ALLOC(cudaMallocAsync(&totals, sizeof(int) * 8, st));
  k_pair_count<<<nblk, kPairBlock, 0, st>>>(nsh, ao.l, ao.atom, ao.ex, ao.nbase, d_coords, thr,
                                           counts);
  RIS_CHECK_LAUNCH();
  k_pair_scan<<<1, 32, 0, st>>>(nblk, counts, offs, totals);
  RIS_CHECK_LAUNCH();
  int h_tot[8];
  RIS_CUDA(cudaMemcpyAsync(h_tot, totals, sizeof(h_tot), cudaMemcpyDeviceToHost, st));
  RIS_CUDA(cudaStreamSynchronize(st));
  int n = 0;
  pl.class_off[0] = 0;
  for (int k = 0; k < 6; k++) {
    n += h_tot[k];
    pl.class_off[k + 1] = n;
  }
  pl.npair = n;
  RIS_ALLOC(cudaMallocAsync((void**)&pl.a, sizeof(int) * std::max(n, 1), st));
  RIS_ALLOC(cudaMallocAsync((void**)&pl.b, sizeof(int) * std::max(n, 1), st));
  k_pair_scatter<<<nblk, kPairBlock, 0, st>>>(nsh, ao.l, ao.atom, ao.ex, ao.nbase, d_coords,
                                             thr, offs, pl.a, pl.b);
  RIS_CHECK_LAUNCH();
  RIS_CUDA(cudaFreeAsync(counts, st));
  RIS_CUDA(cudaFreeAsync(offs, st));
  RIS_CUDA(cudaFreeAsync(totals, st));
}

void free_pairs(PairList& pl, cudaStream_t st) {
  if (pl.a) cudaFreeAsync(pl.a, st);
  if (pl.b) cudaFreeAsync(pl.b, st);
  pl.a = pl.b = nullptr;
  pl.npair = 0;
}

// ------------------------------------------------------------------ dispatch
template <int LA, int LB, int LC>
static void launch_int3c(const ShellSet& ao, const ShellSet& aux, const PairList& pl,
                         const double* xyz, const double* tab, int nJ, int nK, double* TJ,
                         double* TK, const long long* poff, cudaStream_t st) {
  const int cls = LA * (LA + 1) / 2 + LB;
  const int p0 = pl.class_off[cls], np = pl.class_off[cls + 1] - p0;
  const int nax = (int)aux.by_l[LC].size();
  if (np == 0 || nax == 0) return;
  const long long nt = (long long)np * nax;
  k_int3c<LA, LB, LC><<<(unsigned)cdiv(nt, 128), 128, 0, st>>>(
      pl.a, pl.b, p0, np, aux.d_by_l[LC], nax, ao.atom, ao.off, ao.ex, ao.nbase, aux.atom, aux.ex,
      aux.nbase, aux.jmap, aux.kmap, xyz, tab, ao.nfun, nJ, nK, TJ, TK, poff, aux.off);
  RIS_CHECK_LAUNCH();
}

template <int LA, int LB, int LC, class T>
static void launch_int3c_deriv(const ShellSet& ao, const ShellSet& aux, const PairList& pl,
                               const double* xyz, const double* tab, T* D, cudaStream_t st) {
  const int cls = LA * (LA + 1) / 2 + LB;
  const int p0 = pl.class_off[cls], np = pl.class_off[cls + 1] - p0;
  const int nax = (int)aux.by_l[LC].size();
  if (np == 0 || nax == 0) return;
  const long long nt = (long long)np * nax;
  k_int3c_deriv<LA, LB, LC, T><<<(unsigned)cdiv(nt, 128), 128, 0, st>>>(
      pl.a, pl.b, p0, np, aux.d_by_l[LC], nax, ao.atom, ao.off, ao.ex, ao.nbase, aux.atom,
      aux.off, aux.ex, aux.nbase, xyz, tab, ao.nfun, aux.nfun, D);
  RIS_CHECK_LAUNCH();
}

#define RIS_FOR_CLASSES(M, ...)   \
  M<0, 0, 0>(__VA_ARGS__);        \
  M<1, 0, 0>(__VA_ARGS__);        \
  M<1, 1, 0>(__VA_ARGS__);        \
  M<2, 0, 0>(__VA_ARGS__);        \
  M<2, 1, 0>(__VA_ARGS__);        \
  M<2, 2, 0>(__VA_ARGS__);        \
  M<0, 0, 1>(__VA_ARGS__);        \
  M<1, 0, 1>(__VA_ARGS__);        \
  M<1, 1, 1>(__VA_ARGS__);        \
  M<2, 0, 1>(__VA_ARGS__);        \
  M<2, 1, 1>(__VA_ARGS__);        \
  M<2, 2, 1>(__VA_ARGS__);        \
  M<0, 0, 2>(__VA_ARGS__);        \
  M<1, 0, 2>(__VA_ARGS__);        \
  M<1, 1, 2>(__VA_ARGS__);        \
  M<2, 0, 2>(__VA_ARGS__);        \
  M<2, 1, 2>(__VA_ARGS__);        \
  M<2, 2, 2>(__VA_ARGS__);

void int3c(const ShellSet& ao, const ShellSet& aux, const PairList& pl, const double* xyz, int nJ,
           int nK, double* TJ, double* TK, cudaStream_t st) {
  int dev;
  RIS_CUDA(cudaGetDevice(&dev));
  const double* tab = boys_table_device(dev);
  prof_begin(kProfInt3c, st);
  RIS_FOR_CLASSES(launch_int3c, ao, aux, pl, xyz, tab, nJ, nK, TJ, TK, nullptr, st)
  prof_end(kProfInt3c, st, (double)pl.npair * aux.n);
}

void int3c_pairs(const ShellSet& ao, const ShellSet& aux, const PairList& pl, const double* xyz,
                 const long long* poff, double* Ts, cudaStream_t st) {
  int dev;
  RIS_CUDA(cudaGetDevice(&dev));
  const double* tab = boys_table_device(dev);
  prof_begin(kProfInt3c, st);
  RIS_FOR_CLASSES(launch_int3c, ao, aux, pl, xyz, tab, aux.nfun, 0, Ts, nullptr, poff, st)
  prof_end(kProfInt3c, st, (double)pl.npair * aux.n);
}

template <class T>
void int3c_deriv(const ShellSet& ao, const ShellSet& aux, const PairList& pl, const double* xyz,
                 T* D, cudaStream_t st) {
  int dev;
  RIS_CUDA(cudaGetDevice(&dev));
  const double* tab = boys_table_device(dev);
  prof_begin(kProfInt3cDeriv, st);
  RIS_FOR_CLASSES(launch_int3c_deriv, ao, aux, pl, xyz, tab, D, st)
  prof_end(kProfInt3cDeriv, st, (double)pl.npair * aux.n);
}
template void int3c_deriv<double>(const ShellSet&, const ShellSet&, const PairList&, const double*,
                                  double*, cudaStream_t);
template void int3c_deriv<float>(const ShellSet&, const ShellSet&, const PairList&, const double*,
                                 float*, cudaStream_t);

void int2c(const ShellSet& aux, const double* xyz, double* M, double* dM, cudaStream_t st) {
  int dev;
  RIS_CUDA(cudaGetDevice(&dev));
  const double* tab = boys_table_device(dev);
  const int n = aux.n;
  k_int2c<<<cdiv((long long)n * n, 128), 128, 0, st>>>(n, aux.atom, aux.l, aux.off, aux.ex,
                                                        aux.nbase, xyz, tab, aux.nfun, M, dM);
  RIS_CHECK_LAUNCH();
}

}  // namespace ris

// Boys-function probe used by the parity tests: out[i] = F_{m[i]}(T[i]),
// m[i] <= 9, all pointers on the current device.
extern "C" int ris_debug_boys(int n, const int* m, const double* T, double* out) {
  try {
    int dev;
    RIS_CUDA(cudaGetDevice(&dev));
    const double* tab = ris::boys_table_device(dev);
    ris::k_boys_probe<<<ris::cdiv(n, 128), 128>>>(n, m, T, tab, out);
    RIS_CUDA(cudaGetLastError());
    RIS_CUDA(cudaDeviceSynchronize());
    return 0;
  } catch (const ris::Error& e) {
    fprintf(stderr, "ris_debug_boys: %s\n", e.msg.c_str());
    return (int)e.code;
  }
}
