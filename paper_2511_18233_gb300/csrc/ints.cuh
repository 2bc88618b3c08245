// Integral engine: shell data, screened pair list, 2c/3c integrals and their
// first derivatives over uncontracted cartesian primitives.
#pragma once
#include <vector>

#include "common.cuh"

namespace ris {

// Shell arrays on the device (structure of arrays).
struct ShellSet {
  int n = 0;          // number of shells
  int nfun = 0;       // number of functions
  int* atom = nullptr;
  int* l = nullptr;
  int* off = nullptr;        // first function of each shell
  double* ex = nullptr;      // exponent
  double* nbase = nullptr;   // (2a/pi)^(3/4) (4a)^(l/2)
  int* jmap = nullptr;       // auxiliary only: function offset in the J set or -1
  int* kmap = nullptr;       // auxiliary only: function offset in the K set or -1
  std::vector<int> h_atom, h_l, h_off, h_jmap, h_kmap;
  std::vector<double> h_ex;
  std::vector<int> by_l[kMaxLAux + 1];  // auxiliary shells grouped by l
  int* d_by_l[kMaxLAux + 1] = {nullptr, nullptr, nullptr};
  int* fun_atom = nullptr;   // atom of each function
};

// Screened shell-pair list, canonical order la >= lb, grouped by class
// id = la(la+1)/2 + lb.
struct PairList {
  int npair = 0;
  int* a = nullptr;
  int* b = nullptr;
  int class_off[7] = {0, 0, 0, 0, 0, 0, 0};
};

// Boys table F_m(k dT), m = 0..kBoysM, k = 0..kBoysNT-1 (device, [k][m]).
const double* boys_table_device(int device);

void build_pairs(const ShellSet& ao, const double* d_coords, double thr, PairList& pl,
                 void* scratch_pool, cudaStream_t st);
void free_pairs(PairList& pl, cudaStream_t st);

// (mu nu|P) for the auxiliary union set, written to TJ[mu][nu][PJ] and
// TK[mu][nu][PK] (both orderings of mu, nu).  The buffers must be zeroed.
void int3c(const ShellSet& ao, const ShellSet& aux, const PairList& pl, const double* d_coords,
           int nJ, int nK, double* TJ, double* TK, cudaStream_t st);

// Screened-pair storage of (mu nu|P): for each shell pair ip of the list
// (canonical order), its na x nb function pairs are rows poff[ip] + ia * nb
// + ib of Ts [rows][aux.nfun] (mu of the pair's first shell, nu of its
// second; P in the auxiliary set's own function order).
void int3c_pairs(const ShellSet& ao, const ShellSet& aux, const PairList& pl, const double* xyz,
                 const long long* poff, double* Ts, cudaStream_t st);

// D[x][mu][nu][P] = d(mu nu|P)/dA_x with A the centre of mu (union auxiliary
// set, P fastest), computed in FP64 and stored as T (double or float).
// Zeroed by the caller.
template <class T>
void int3c_deriv(const ShellSet& ao, const ShellSet& aux, const PairList& pl,
                 const double* d_coords, T* D, cudaStream_t st);

// M[P][Q] = (P|Q) over the union set, and dM[x][P][Q] = d(P|Q)/dP_x.
void int2c(const ShellSet& aux, const double* d_coords, double* M, double* dM, cudaStream_t st);

}  // namespace ris
