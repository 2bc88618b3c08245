// TDDFT-ris engine state and stages.
#pragma once
#include <map>
#include <string>
#include <vector>

#include "gemm_emu.cuh"
#include "gemm_tc.cuh"
#include "ints.cuh"
#include "la.cuh"

namespace ris {

// Device buffer owned by the context (stream-ordered, tracked).
struct DBuf {
  double* p = nullptr;
  size_t n = 0;
  cudaStream_t st = nullptr;
  MemTrack* tr = nullptr;
  void ensure(size_t count, cudaStream_t s);
  void release();
  ~DBuf() { release(); }
};

// Stream-ordered temporary (cudaMallocAsync / cudaFreeAsync from the
// device's memory pool, which the context keeps from releasing), optionally
// zero-filled.
template <class T>
struct SBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t st = nullptr;
  MemTrack* tr = nullptr;
  SBuf() = default;
  SBuf(size_t count, cudaStream_t s, bool zero = false) { ensure(count, s, zero); }
  void ensure(size_t count, cudaStream_t s, bool zero = false) {
    if (p && count <= n) return;
    release();
    st = s;
    if (count == 0) count = 1;
    p = (T*)dev_alloc(count * sizeof(T), st, &tr);
    n = count;
    if (zero) RIS_CUDA(cudaMemsetAsync(p, 0, count * sizeof(T), st));
  }
  void release() {
    if (p) dev_free(p, n * sizeof(T), st, tr);
    p = nullptr;
    n = 0;
  }
  ~SBuf() { release(); }
  SBuf(const SBuf&) = delete;
  SBuf& operator=(const SBuf&) = delete;
};

// FP32 device buffer (zero-filled when (re)allocated).
struct FBuf {
  float* p = nullptr;
  size_t n = 0;
  cudaStream_t st = nullptr;
  MemTrack* tr = nullptr;
  void ensure(size_t count, cudaStream_t s);
  void release();
  ~FBuf() { release(); }
};

// The context's stream; a base class so that it outlives every buffer
// member, whose stream-ordered frees are queued on it.
struct StreamOwner {
  cudaStream_t st = nullptr;
  bool own_stream = false;
  cudaStream_t st2 = nullptr;  // low-priority side stream (derivative integrals)
  cudaStream_t st3 = nullptr;  // side stream: the pair list to the host, the metric factors
  cudaEvent_t evP = nullptr;   // the pair list is built
  cudaEvent_t evC = nullptr;   // its host copy is done
  cudaEvent_t evM = nullptr;   // the metric factors are done (st3)
  int* pin = nullptr;          // pinned host copy of the pair list
  size_t pin_n = 0;
  ~StreamOwner() {
    if (st3) cudaStreamSynchronize(st3);
    if (pin) cudaFreeHost(pin);
    if (evP) cudaEventDestroy(evP);
    if (evC) cudaEventDestroy(evC);
    if (evM) cudaEventDestroy(evM);
    if (st3) cudaStreamDestroy(st3);
    if (st2) cudaStreamDestroy(st2);
    if (own_stream && st) cudaStreamDestroy(st);
  }
};

struct Engine;

// Coulomb-exact preconditioner (definition and formula in engine.cu).
struct CoulPrecond {
  SBuf<double> dinv, capinv, pY, pZ, pP;
  // mixed precision (when small): hi/lo splits of B^J as [ia][P] and
  // [P][ia] and of the work vectors, for 3xTF32 applications
  SBuf<float> Bh, Bl, BTh, BTl, Th, Tl, Zh, Zl;
  bool tc = false;
  double f = 2.0;
  void setup(Engine& e, bool shifted, double f, int nmax);
  // T[j] = M^-1 R[idx ? idx[j] : j], j < nt <= nmax
  void apply(Engine& e, const double* R, const int* idx, int nt, double* T);
};

struct Engine : StreamOwner {
  ris_options opt{};
  int device = 0;
  MemTrack mem;
  mutable std::string err;  // last error message (also set by the const statistics call)
  int stage = 0;  // 0 created, 1 aux built, 2 B built, 3 excited

  // geometry / basis
  int natm = 0;
  DBuf xyz;
  ShellSet ao, aux;   // aux = union of the J and K sets, K functions first
  int nJ = 0, nK = 0, nU = 0;
  std::vector<int> h_jU, h_kU;  // J / K function -> union function
  std::vector<int> h_kJ;        // K function -> J function (-1: none)
  int* d_jU = nullptr;
  int* d_kU = nullptr;
  int* d_kJ = nullptr;  // K function -> J column, when every K function is also a J function
  // functions of each atom (CSR): AO functions and union auxiliary functions
  SBuf<int> aoPtr, aoList, axPtr, axList;
  PairList pl;
  DBuf TJ, TK;              // (mu nu|P) [mu][nu][P] per set
  DBuf MU, dMU;             // union metric and d/dP_x
  DBuf LJinv, LKinv;        // inverse Cholesky factors
  DBuf D;                   // derivative integrals [3][mu][nu][P_U] (FP64 path)
  FBuf Df;                  // the same in FP32 storage (mixed precision)
  bool have_D = false;
  bool D_pending = false;             // D being computed on st2 (event evD)
  cudaEvent_t evA = nullptr, evD = nullptr;
  int* d_info = nullptr;

  // MO data
  int nao = 0, nmo = 0, nocc = 0, nvir = 0;  // active sizes (after mo_window)
  int first_occ = 0;                           // first active occupied MO of the input
  DBuf C, eps, de;
  DBuf BJ;        // [ov][RJ]
  DBuf BKoo;      // [i][j][R]
  DBuf BKvvD;     // [b][R][a] (Davidson layout)
  DBuf BKovR;     // [R][i][a] (RPA)
  DBuf cKovP;     // c^K_ov as [P][i][a] (RPA)
  DBuf cKoo, cKvv, cKov;  // fitting coefficients c = B L^-1, [p][q][P]

  // mixed precision (3xTF32) operands: hi/lo FP32 splits
  FBuf BooH, BooL;  // B^K_oo as [i][R][j] (ld ld4(nocc))
  FBuf BvvH, BvvL;  // B^K_vv as [a][R][b] (b padded to ld4(nvir))
  FBuf XtH, XtL;    // amplitudes transposed [vec][b][j]
  FBuf YH, YL;      // [vec][i][R][b] = sum_j B^K_oo[R][i][j] X[vec][j][b]
  FBuf cvvH, cvvL;  // c^K_vv as [(P,b)][a] (a padded)
  DBuf cKooP;       // c^K_oo as [P][i][k] (FP64)
  FBuf cooH, cooL;  // c^K_oo as [(P,k)][i] (i padded)
  FBuf CoH, CoL;    // C_o as [mu][j] (j padded)
  FBuf CvH, CvL;    // C_v as [mu][a] (a padded)
  int* d_tcerr = nullptr;

  // excitations
  int nstates = 0;
  DBuf omega, X, Y;
  std::vector<double> h_omega;

  // screened partners of each AO function (CSR over the screened shell-pair
  // list), the nu range of the derivative contractions
  SBuf<int> nbPtr, nbCol;
  int nbAvg = 1;
  std::vector<int> h_pa, h_pb;  // the screened shell pairs on the host
  void partners_from_host_pairs();  // nbPtr / nbCol from h_pa / h_pb
  // streamed form (large systems): three-centre integrals on the screened
  // function pairs only, mixed with the metric factors there; auxiliary
  // blocks for the MO transforms and the derivative integrals
  bool streamed = false;
  long long nfp = 0;        // function pairs of the screened shell-pair list
  SBuf<long long> pOff;     // first function-pair row of each shell pair
  SBuf<int> fpMu, fpNu;     // the two AO functions of each function pair
  DBuf BJao, BKao;          // [fp][R]: sum_P (mu nu|P) (L_X^-1)_RP on the screened pairs
  std::vector<int> blkU0, blkW, blkWK;  // auxiliary blocks: first union function, width, K part
  std::vector<ShellSet> auxBlk;        // the blocks' shells with block-local offsets
  int nKsh = 0;                         // K shells (the first nKsh union shells)

  // work
  DBuf w1, w2, w3, w4, w5, w6, w7, w8;
  double stats[16] = {0};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  ~Engine();
  // release every device buffer (the context returns to its created state)
  void trim();
  void build_aux(int natm, const double* coords, int nshell, const ris_shell* ao,
                 int nJs, const ris_shell* auxJ, int nKs, const ris_shell* auxK);
  void build_B(int nao, int nmo, int nocc, const double* C, const double* mo_energy);
  void excite(int nstates, double* omega, double* X, double* Y, const double* guess = nullptr);
  // numerators dE_IJ/dR for pairs, [npair][natm][3] into out (host or device)
  void pair_derivs(int npair, const int* pairs, int nx, const double* X_in, const double* Y_in,
                   double* out_dev);
  void ensure_D();
  void start_D(cudaStream_t s);  // derivative integrals on stream s
  void join_D();                 // make st wait for a pending D
  void apply(int nvec, const double* X, double* out, double* out2);

  // helpers
  void apply_A_tda(const double* Xin, int nvec, double* out);
  void apply_A_mixed(const double* Xin, int nvec, double* out);
  void apply_exchange_mixed(const double* Z, int nvec, double* out, double alpha, double beta);
  void prepare_mixed();
  void build_Kvv_tc(double* out);
  void coulomb_emu(double* H, double* W);  // H [nu][i][P], W [i][a][P] (mixed form)
  // C = A B^T, element (r, k) of A at A[r rsA + k ksA] (B likewise), as an
  // FP64-accurate product on the tensor cores
  void emu_abt(int M, int N, int K, const double* A, long long rsA, long long ksA, const double* B,
               long long rsB, long long ksB, const EmuEpilogue& ep);
  // exchange part of Gamma / Omega for one (U,V) pair with weight f (3xTF32);
  // US/VS: splits of U, V [i][a]; WU/WV: [Q^T | C_o] splits of U and V;
  // Gamma accumulated in FP64 (Gam) or, when Gam32 is given, written in FP32
  // (overwritten: the caller's only exchange term)
  void gamma_K_mixed(const float* USh, const float* USl, const float* VSh, const float* VSl,
                     const float* WUh, const float* WUl, const float* WVh, const float* WVl,
                     double f, double* Gam, float* Gam32, double* Om);
  // ok != nullptr: a mixed-precision run that stalls above the tolerance
  // returns its current vectors with *ok = false instead of failing
  void dav_core(int ns, const double* guess, int nguess, bool mixed, double tol,
                bool augment = false, bool* ok = nullptr);
  void apply_ApB_AmB(const double* Zin, int nvec, double* outP, double* outM);
  void davidson_tda(int ns, const double* guess = nullptr);
  void davidson_rpa(int ns);
  // ris Z-vector solve (A+B) Z = rhs for nr right-hand sides (PCG)
  void zvector(int nr, const double* rhs, double* Z);
  void ensure_Kov();
  // time-derivative couplings T[g] = d_g . v (nac [npair][natm][3], vel [natm][3])
  void time_coupling(int npair, const double* nac, const double* vel, double* T);
  // phases of the current states against the previous step (five dominant determinants)
  void phase_align(int ns, const double* Xprev, int* sign, double* Xout);
  // exchange (ij|ab) and (ib|ja) contractions of nvec vectors: K1, K2 [nvec][nov]
  void exchange_terms(const double* Z, int nvec, double* K1, double* K2, bool mixed);
  // streamed form
  bool want_streamed(int nao_) const;
  void setup_streamed();
  void build_B_streamed();
  void pair_derivs_streamed(int npair, const int* pairs, int nsu, const std::vector<int>& su,
                            const std::map<int, int>& slot, const double* Xa, double* out);
  int block_width(double bytes_per_function) const;
};

// n doubles from a host or device pointer into host memory
void copy_to_host(double* dst, const double* src, size_t n, cudaStream_t st);

// out[g][k] = num[g][k] / den[g]
void divide_pairs(double* out, const double* num, const double* den, int npair, int per,
                  cudaStream_t st);

}  // namespace ris
