/*
 * ris.h — C ABI of the GB300 (sm_103a) TDDFT-ris engine.
 *
 * The engine evaluates the minimal-auxiliary-basis ("ris") response kernel
 * of arXiv:2511.18233 and its explicit nuclear derivatives:
 *
 *   - the ris two-electron kernel, Eq. (g_modified) of Sec. 2.2:
 *       g^ris_{pq,sr} = sum_AB (pq|A)(M^-1)_AB(B|sr) - c_x sum_AB (pr|A)(M^-1)_AB(B|sq),
 *     M_AB = (A|B), with separate Coulomb-fitting (J) and exchange-fitting (K)
 *     auxiliary sets (Sec. 2.2; Sec. 4 uses s+p for J and s for K);
 *   - the Casida problem, Eqs. (casida), (A_matrix), (B_matrix), with the pure
 *     XC kernel dropped (Eq. (ris)); closed-shell singlet, so
 *       A_ia,jb = (e_a - e_i) d_ij d_ab + 2 (ia|jb)_J - c_x (ij|ab)_K,
 *       B_ia,jb = 2 (ia|jb)_J - c_x (ib|ja)_K;
 *     TDA is the same path with Y = 0 (Sec. 3);
 *   - the integral-derivative terms <g^{ris,(xi)}; Gamma_II> and
 *     <g^{ris,(xi)}; Gamma_IJ>/(E_J - E_I) of Eqs. (gI_xi_ris) and
 *     (gIJ_xi_ris), with the RI derivative formula closing Sec. 2.2 and
 *     Gamma_IJ = {R_I^S,R_J^S} + {L_I^A,L_J^A} (Appendix A).
 *
 * The gradient returned is the derivative of the pair energy
 *     E_IJ = 1/2 [R_I (A+B) R_J + L_I (A-B) L_J],  R = X+Y, L = X-Y,
 * with respect to the nuclear coordinates at fixed MO coefficients, orbital
 * energies and amplitudes; g_I = dE_II/dR (Eq. (gradient)) and the
 * derivative coupling g_IJ = (dE_IJ/dR)/(omega_J - omega_I) (Eq. (fo-nacme)).
 *
 * Conventions
 *   - Units: bohr and Hartree; gradients in Hartree/bohr, couplings in 1/bohr.
 *   - Every shell is one uncontracted cartesian primitive, each component
 *     normalised to <chi|chi> = 1; components in lexicographic order
 *     (p: x,y,z; d: xx,xy,xz,yy,yz,zz).  AO functions are numbered shell by
 *     shell in the order given.
 *   - All matrices are row-major.  Amplitudes are [nstate][nocc][nvir] (the
 *     transpose of the paper's vir x occ X_ai).
 *   - Array arguments may be host or device pointers.  A device pointer must
 *     live on the context's device; it is read or written in stream order on
 *     the context's stream.  The library tells the two apart with
 *     cudaPointerGetAttributes.
 *
 * Ownership and errors
 *   - The caller owns every argument buffer; the context copies what it keeps
 *     and owns all device memory it allocates.
 *   - Every call returns a ris_status.  On error the outputs are untouched and
 *     ris_last_error() returns a message; the one exception is ris_nac, which
 *     still writes the requested numerators when it returns
 *     RIS_ERR_DEGENERATE (the couplings themselves are untouched).  Calls made
 *     out of order (aux -> B -> excite -> gradient/nac) return RIS_ERR_STATE.
 *   - One context per stream; contexts share no state.
 */
#ifndef RIS_H_
#define RIS_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ris_ctx ris_ctx;

typedef enum {
  RIS_OK = 0,
  RIS_ERR_ARG = -1,            /* invalid argument */
  RIS_ERR_OOM = -2,            /* device allocation failed or over mem_budget */
  RIS_ERR_METRIC_NOT_PD = -3,  /* auxiliary metric not positive definite */
  RIS_ERR_NOT_CONVERGED = -4,  /* Davidson hit max_iter */
  RIS_ERR_CUDA = -5,           /* CUDA runtime error */
  RIS_ERR_TIMEOUT = -6,        /* a host wait exceeded its limit */
  RIS_ERR_STATE = -7,          /* call order violated */
  RIS_ERR_DEGENERATE = -8      /* |omega_J - omega_I| too small for a coupling */
} ris_status;

enum { RIS_FP64 = 0, RIS_MIXED = 1 };

typedef struct {
  int precision;      /* RIS_FP64, or RIS_MIXED: the (ab|P)_K half transforms of the
                         B-tensor build, the exchange part of every Davidson product and
                         the exchange part of Gamma as 3xTF32 tensor-core GEMMs with FP32
                         accumulation (integrals, metric Cholesky, the Coulomb part,
                         orthogonalisation, subspace eigenproblem and the gradient
                         accumulation stay FP64) */
  int rpa;            /* 0: TDA (Y = 0), 1: full RPA (X, Y) */
  double cx;          /* fraction of exact exchange c_x (Eq. g_integral); default 0.25 */
  double conv_tol;    /* Davidson residual 2-norm per state; default 1e-10 */
  int max_iter;       /* Davidson iterations; default 100 */
  int max_subspace;   /* Davidson subspace size before restart; 0 = automatic: max(initial
                         block + 2 nstates, 8 nstates), 4 nstates instead of 8 in the mixed
                         phase when nocc*nvir <= 2^20 (TDA) */
  double screen_thr;  /* shell-pair screening threshold; default 1e-14 */
  size_t mem_budget;  /* device bytes the context may hold; 0 = no limit */
  int occ_block;      /* occupied orbitals per block of the exchange part of the Davidson
                         products; 0 = automatic (all when they fit) */
  void* cuda_stream;  /* cudaStream_t to run on; NULL = the context makes one */
  int device;         /* CUDA device ordinal */
  int profile;        /* 1: time the kernel classes this context launches with CUDA events on
                         its streams (see ris_get_stats; other contexts are not counted) */
  double mixed_tol;   /* RIS_MIXED: residual tolerance of the 3xTF32 Davidson phase; default 1e-6.
                         When the 3xTF32 products stall above it (eight iterations without a
                         10% drop of the largest residual, within 100x the tolerance), TDA
                         continues with FP64 products to the same tolerance (not available in
                         the streamed form, which keeps no FP64 B^K_vv) */
  int refine;         /* RIS_MIXED: 1 = continue with FP64 products to conv_tol (the B
                         tensors are then built in FP64 throughout); default 0 */
  int precond;        /* TDA Davidson preconditioner: 0 (default) = (D - s + 2 B^J B^J^T)^-1
                         applied exactly (Woodbury) with one shift s just below the smallest
                         orbital-energy difference; 1 = diagonal (D - omega_k)^-1 per state */
  double mo_window;   /* > 0: keep only occupied MOs with e_i >= e_HOMO - mo_window and virtual
                         MOs with e_a <= e_LUMO + mo_window (Hartree; orbital energies sorted
                         within each block); amplitudes are then [nocc_act][nvir_act]
                         (ris_get_mo_window).  0 (default): all MOs */
  int deriv_prefetch; /* 1 (default): ris_build_aux also starts the derivative integrals on a
                         second, low-priority stream, overlapping the B build and the
                         Davidson; the first gradient / coupling call waits for them.
                         0: computed by the first derivative call */
  int emu_f64;        /* mixed precision: 1 (default) runs the Coulomb B transforms
                         (the two MO transforms of (mu nu|P)_J) as FP64-accurate products
                         on the FP16 tensor cores by exact operand splitting; 0: FP64 */
  int eig_fp32;       /* mixed precision: 1 solves the Davidson subspace eigenproblem in FP32
                         (FP64 Rayleigh quotients, close pairs and restarts re-orthonormalised
                         in FP64, back to FP64 if the residuals stall); 0 (default): FP64 */
  int stream;         /* streamed form for systems whose dense AO three-index tensors do not
                         fit (TDA only): the three-centre integrals are kept only on the
                         screened shell pairs and mixed with the metric factors there, the MO
                         transforms run over blocks of auxiliary functions, the exchange part
                         of each Davidson product over blocks of occupied orbitals
                         (occ_block), and the gradient regenerates the derivative integrals
                         per block of auxiliary functions instead of storing them.
                         0 (default): automatic (streamed when the dense integrals and
                         derivative integrals would take more than a third of the device
                         memory or of mem_budget); 1: always; -1: never */
  int stream_block;   /* streamed form: auxiliary functions per block; 0 = automatic */
  int subspace_ff;    /* mixed precision: 1 (default) forms the Davidson Ritz vectors X = S V,
                         A X = S (A V) and the Coulomb part of the A products as double-FP32
                         products on the FP32 pipe (error per element at most about 3e-11 of
                         sum |a||b|, see ris_debug_gemm_ff); the orthogonalisation and the
                         projected matrix V^T A V stay FP64.  0: all FP64 */
} ris_options;

typedef struct {
  int atom;        /* index into the coordinate array */
  int l;           /* angular momentum: AO 0..2, auxiliary 0..1 */
  double exponent; /* Gaussian exponent (bohr^-2) */
} ris_shell;

/* Fill *opt with the defaults listed above. */
ris_status ris_options_default(ris_options* opt);

/* Create a context on opt->device.  *out receives the handle. */
ris_status ris_create(ris_ctx** out, const ris_options* opt);

/*
 * Geometry and basis (Sec. 2.2: the ris auxiliary set is one Gaussian per
 * angular-momentum component per atom).  coords: [natm][3] bohr.  ao: the AO
 * shells; auxJ / auxK: Coulomb- and exchange-fitting auxiliary shells.
 * Builds the screened shell-pair list, the three-centre integrals (mu nu|P)
 * and the metric Cholesky factor M = L L^T of each auxiliary set.
 * Invalidates any earlier B tensors and excitations.
 * Errors: RIS_ERR_ARG (bad shell, l out of range, atom index out of range),
 * RIS_ERR_METRIC_NOT_PD (singular metric, e.g. duplicate atoms).
 */
ris_status ris_build_aux(ris_ctx* ctx, int natm, const double* coords, int nshell,
                         const ris_shell* ao, int nJ, const ris_shell* auxJ, int nK,
                         const ris_shell* auxK);

/*
 * MO data and the B tensors B^X_{pq,R} = sum_P (pq|P) (L_X^-T)_PR (RI of
 * Eq. (g_modified)): B^J over the ov block and B^K over the oo and vv blocks
 * (plus ov for RPA).  C: [nao][nmo] row-major, occupied columns first;
 * mo_energy: [nmo].  nmo <= nao (fewer MOs than AOs when near-dependent AO
 * combinations were dropped); 0 < nocc < nmo.
 */
ris_status ris_build_B(ris_ctx* ctx, int nao, int nmo, int nocc, const double* C,
                       const double* mo_energy);

/*
 * Lowest nstates excitation energies by Davidson on the ris A (TDA) or on the
 * Casida problem (RPA), Eq. (casida).  omega: [nstates] Hartree.  X, Y:
 * [nstates][nocc][nvir] or NULL (Y is written only for RPA).  Normalisation:
 * sum X^2 = 1 (TDA), sum X^2 - Y^2 = 1 (RPA); each state's sign makes its
 * largest-magnitude X element positive.
 * Errors: RIS_ERR_NOT_CONVERGED after max_iter (outputs untouched).
 */
ris_status ris_excite(ris_ctx* ctx, int nstates, double* omega, double* X, double* Y);

/*
 * As ris_excite (TDA), but the Davidson search starts from the nstates given
 * vectors X_guess [nstates][nocc][nvir] (host or device) instead of unit
 * vectors — for instance the amplitudes of the previous step of a
 * trajectory.  The guesses need not be normalised but must be linearly
 * independent (RIS_ERR_ARG otherwise).  With the rpa option the guess is
 * ignored and the search starts cold.
 */
ris_status ris_excite_guess(ris_ctx* ctx, int nstates, const double* X_guess, double* omega,
                            double* X, double* Y);

/*
 * Phase tracking along a trajectory (Sec. 2, phase determination for
 * derivative couplings along a geometric path): for each of the first
 * nstates states of the last ris_excite, the overlap with the previous
 * step's state over its five most dominant determinants (the five largest
 * |X_prev| elements, ties by index; MOs common to both steps) decides the
 * sign, and a negative overlap flips the state's X (and Y).  Later
 * ris_gradient / ris_nac calls without explicit amplitudes use the aligned
 * phases.  X_prev: [nstates][nocc][nvir] (host or device); sign: [nstates]
 * +1 / -1 (host or device, may be NULL); X_out: aligned X (may be NULL).
 */
ris_status ris_phase_align(ris_ctx* ctx, int nstates, const double* X_prev, int* sign,
                           double* X_out);

/*
 * Time-derivative couplings of surface hopping (Sec. 4: the hopping
 * probabilities use T_IJ = g_IJ . v, the derivative coupling projected on
 * the nuclear velocities): T[g] = sum_{A,x} nac[g][A][x] velocity[A][x] for
 * npair couplings.  nac: [npair][natm][3] (1/bohr, e.g. from ris_nac);
 * velocity: [natm][3] (bohr per atomic time unit); T: [npair].  Host or
 * device pointers.  Needs ris_build_aux (for natm).
 */
ris_status ris_time_coupling(ris_ctx* ctx, int npair, const double* nac, const double* velocity,
                             double* T);

/*
 * The ris-approximated Z-vector solve: (A + B) Z = rhs (Eq. Z_vector, with
 * the ris kernel of Eq. ris in A + B — the solver of the section "Ris
 * approximation for Z-vector Solver"), for nrhs <= 64 right-hand sides at
 * once.  rhs, Z: [nrhs][nocc][nvir] (host or device).  Preconditioned
 * conjugate gradients (A + B is symmetric positive definite for a stable
 * ground state); preconditioner: orbital-energy differences plus the exact
 * Coulomb part 4 B^J B^J^T (Woodbury).  Converged when every residual
 * satisfies |rhs - (A+B) Z| <= tol |rhs| with tol = conv_tol (RIS_FP64) or
 * max(conv_tol, mixed_tol) (RIS_MIXED, 3xTF32 (ij|ab) products); otherwise
 * RIS_ERR_NOT_CONVERGED after max_iter iterations.  Stats [4] products, [5]
 * iterations, [7] largest relative residual.  Works for TDA and RPA contexts
 * (the (ib|P) block is built on first use).
 */
ris_status ris_zvector(ris_ctx* ctx, int nrhs, const double* rhs, double* Z);

/*
 * The response operator applied to nvec vectors (the Davidson product of
 * Eqs. (A_matrix)/(B_matrix) with the ris kernel): TDA: out = A X; RPA
 * (rpa option set): out = (A+B) X followed by out2 = (A-B) X.
 * X, out, out2: [nvec][nocc][nvir]; out2 must be NULL for TDA.
 * Requires ris_build_B.
 */
ris_status ris_apply(ris_ctx* ctx, int nvec, const double* X, double* out, double* out2);

/*
 * Excited-state gradients g_I = dE_II/dR (Eq. (gI_xi_ris), integral-derivative
 * term) for the n states listed in states[] (0-based).  If X_in is NULL the
 * amplitudes of the last ris_excite are used and states index them;
 * otherwise X_in (and Y_in for RPA, NULL for TDA) hold nx states
 * [nx][nocc][nvir] and states index those.  grad: [n][natm][3] Hartree/bohr.
 */
ris_status ris_gradient(ris_ctx* ctx, int n, const int* states, int nx, const double* X_in,
                        const double* Y_in, double* grad);

/*
 * Derivative couplings g_IJ = (dE_IJ/dR)/(omega_J - omega_I) (Eqs. (fo-nacme),
 * (gIJ_xi_ris), integral-derivative term) for npair pairs [npair][2].
 * Amplitudes as in ris_gradient; omega_in: [nx] energies for X_in (NULL with
 * X_in NULL).  nac: [npair][natm][3] 1/bohr; numerator (dE_IJ/dR, same
 * shape) may be NULL.  Returns RIS_ERR_DEGENERATE if |omega_J - omega_I| <
 * 1e-8 for a pair (the numerator is still written when requested).
 */
ris_status ris_nac(ris_ctx* ctx, int npair, const int* pairs, int nx, const double* X_in,
                   const double* Y_in, const double* omega_in, double* nac, double* numerator);

/*
 * The active MO range after ris_build_B: occupied MOs first_occ .. nocc-1 and
 * the first nvir_act virtual MOs (all of them without mo_window); the
 * amplitudes of every call are [nocc_act][nvir_act].  Any pointer may be NULL.
 */
ris_status ris_get_mo_window(const ris_ctx* ctx, int* first_occ, int* nocc_act, int* nvir_act);

/* Sizes of the current problem (any pointer may be NULL). */
ris_status ris_get_dims(const ris_ctx* ctx, int* natm, int* nao, int* nocc, int* nauxJ,
                        int* nauxK, int* npairs_screened);

/*
 * Statistics, copied into out[0..n-1] (n <= 34):
 *   [0] aux, [1] B, [2] excite (or Z-vector), [3] gradient/nac: milliseconds
 *       of the last call of each kind (CUDA events on the context's stream);
 *   [4] A-products and [5] Davidson iterations of the last excite (or the
 *   (A+B) products and CG iterations of the last Z-vector solve),
 *   [6] FP64 products of its refinement phase (mixed with refine, or the
 *   FP64 continuation after the 3xTF32 products stalled above mixed_tol), [7] the
 *   largest residual norm |A x - omega x| at its last iteration (TDA);
 *   [15] kernels launched by the library since it was loaded (all contexts);
 *   with the profile option, per kernel class since the previous call:
 *   [16] GEMM ms, [17] GEMM flops, [18] 3c-integral ms, [19] shell triples,
 *   [20] 3c-derivative ms, [21] shell triples, [22] derivative-contraction
 *   ms, [23] its algorithmic bytes, [24] subspace-eigensolver ms, [25] calls,
 *   [26] 3xTF32 tensor-core GEMM ms, [27] its algorithmic flops (one per
 *   multiply-add pair of the product, the three TF32 passes counted once);
 *   [28] device bytes the context holds now, [29] the most it has held
 *   since it was created or last trimmed (its HBM footprint);
 *   [30] FP64-emulating tensor-core GEMM ms, [31] its algorithmic FP64
 *   flops, [32] double-FP32 GEMM ms, [33] its flops (profile option, as
 *   [16]..[27]).
 */
ris_status ris_get_stats(const ris_ctx* ctx, double* out, int n);

/*
 * Release every device buffer the context holds (integrals, B tensors,
 * amplitudes, work space) back to the device's stream-ordered pool and
 * return it to its just-created state; the next call must be
 * ris_build_aux.  Resets the footprint high-water mark (stats [29]).
 * The library allocates from the device's default memory pool in stream
 * order on the context's stream, so several contexts driven from
 * different host threads run concurrently without device-wide
 * synchronisation.  A context must not be used by two threads at once.
 */
ris_status ris_trim(ris_ctx* ctx);

/*
 * Test hook: Boys function F_m(T) = int_0^1 t^{2m} e^{-T t^2} dt as used by
 * the integral kernels (the Coulomb integrals of Eq. (g_modified) reduce to
 * it).  n values; m[i] in 0..9; all three arrays are DEVICE pointers on the
 * current device.  Synchronises the device; returns 0 or a ris_status.
 */
int ris_debug_boys(int n, const int* m, const double* T, double* out);

/*
 * Test hook: C = alpha op(A) op(B) + beta C with the library's FP64 GEMM
 * (the dense contractions of the B-tensor transforms and the Davidson
 * subspace).  Row-major; op(A) is m x k, op(B) is k x n; transA/transB
 * nonzero = transposed operand; lda/ldb/ldc are row strides of the stored
 * arrays.  DEVICE pointers on the current device.  Synchronises the device;
 * returns 0 or a ris_status.
 */
int ris_debug_dgemm(int transA, int transB, int m, int n, int k, double alpha, const double* A,
                    int lda, const double* B, int ldb, double beta, double* C, int ldc);

/*
 * Test hook: lowest k (<= 64) eigenpairs of a symmetric m x m row-major
 * matrix with the device eigensolver of the Davidson subspace problem.
 * H: [m][m], w: [k] ascending, V: [k][m] (row j = eigenvector j); DEVICE
 * pointers on the current device.  Synchronises the device.
 */
int ris_debug_sym_eig(int m, int k, const double* H, double* w, double* V);

/*
 * Test hook: the same with the FP32 form of the eigensolver used by the
 * mixed precision Davidson (m <= 200): FP32 Householder reduction,
 * multisection and inverse iteration; FP64 normalisation and Rayleigh
 * quotients; vectors of eigenvalues closer than 1e-4 ||H|| orthonormalised
 * and rotated onto the Ritz vectors of their span in FP64.  Residuals
 * |H v - w v| of a few FP32 ulps of ||H||.  Returns RIS_ERR_ARG for m > 200.
 */
int ris_debug_sym_eig_f32(int m, int k, const double* H, double* w, double* V);

/*
 * Test hook: C = A . B^T with the library's 3xTF32 tensor-core GEMM (the
 * kernel behind RIS_MIXED).  A: [M][K], B: [N][K], C: [M][N], FP64 DEVICE
 * pointers on the current device (inputs are rounded to FP32 and split).
 * Synchronises the device; returns 0, RIS_ERR_TIMEOUT if a pipeline wait
 * timed out, or another ris_status.
 */
int ris_debug_gemm_tf32x3(int M, int N, int K, const double* A, const double* B, double* C);

/*
 * Test hook: C = A . B^T with the library's FP64-emulating tensor-core GEMM
 * (the kernel behind the Coulomb transforms of RIS_MIXED): both operands are
 * split exactly into ten 6-bit digit slices per row frame (Ozaki's
 * error-free transformation) and multiplied on the FP16 tensor cores with
 * exact FP32 accumulation.  Error per element below about
 * K 2^-54 max_k|A_rk| max_k|B_ck| plus FP64 rounding of the result.
 * A: [M][K], B: [N][K], C: [M][N], FP64 DEVICE pointers on the current
 * device, finite values.  Synchronises the device; returns 0,
 * RIS_ERR_TIMEOUT if a pipeline wait timed out, or another ris_status.
 */
int ris_debug_gemm_f64emu(int M, int N, int K, const double* A, const double* B, double* C);

/*
 * Test hook: C = alpha A op(B) + beta C with the library's double-FP32 GEMM
 * (the kernel behind the mixed form's subspace products): FP64 operands cut
 * into pairs of FP32 numbers, products accumulated by the compensated dot
 * product of Ogita, Rump and Oishi on the FP32 pipe.  Error per element at
 * most about 3e-11 sum_k |A_ik| |op(B)_kj| plus FP64 rounding of the result,
 * for operands of magnitude 2^-74 and above; smaller values keep 24
 * significant bits, below 2^-126 they count as zero; values at or above
 * 2^128 and non-finite values (inf, nan) count as infinite.  A: [M][K]; B: [N][K] if transB else [K][N]; C: [M][N] (read
 * when beta != 0); FP64 DEVICE pointers on the current device.  Shapes:
 * M <= 32 and either K <= 256 with N >= 128, or K >= 512 with N <= 512;
 * *kind (if not null) receives 1 (long-K kernel), 2 (short-K kernel) or 0
 * (shape not handled: RIS_ERR_ARG, nothing launched).  Synchronises the
 * device; returns 0 or a ris_status.
 */
int ris_debug_gemm_ff(int transB, int M, int N, int K, double alpha, const double* A,
                      const double* B, double beta, double* C, int* kind);

/*
 * Allocation-free 3xTF32 GEMM: C = A . B^T computed exactly like
 * ris_debug_gemm_tf32x3, but without allocating device memory.  The paper
 * has no counterpart; this exists for callers that cannot allocate at the
 * point of the call, for example a serving process that hands all free
 * device memory to its own pool up front, or a latency-critical loop where an
 * allocation could block or fail.
 * A: [M][K], B: [N][K], C: [M][N], FP64 DEVICE pointers on the current
 * device; stream: a cudaStream_t or NULL.  Work space comes from one 32 MiB
 * device array that the library reserves on every GPU it is loaded on and
 * holds until the process exits; the call returns RIS_ERR_ARG (with a
 * message on stderr) when 2*(M+N)*ceil4(K) + 64 exceeds its 8 Mi floats.
 * The first call on a device looks the array's address up
 * (cudaGetSymbolAddress), so make that call before any stream capture.
 * Every call uses the same array: calls that overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * The call synchronises the stream; returns 0, RIS_ERR_TIMEOUT if a
 * pipeline wait timed out, or another ris_status.
 */
int ris_gemm_tf32x3_noalloc(int M, int N, int K, const double* A, const double* B, double* C,
                            void* stream);

/*
 * Test hook: measured peak rate of one arithmetic pipe of the current
 * device, the denominator of the roofline fractions of the kernels bound by
 * it.  kind: 0 FP64 FMA, 1 FP32 FMA (SIMT; independent chains on every
 * SM), 2 FP64 mma.sync m16n8k4, 3 tcgen05 kind::tf32 (M 128, N 256, K 8),
 * 4 tcgen05 kind::f16 (M 128, N 256, K 16; one CTA per SM issuing back to
 * back from fixed shared-memory tiles).  Best of reps timed runs after one
 * warm-up run (CUDA events): *tflops in 10^12 flop/s (an FMA or MMA
 * multiply-add counts 2), *ms (may be NULL) the duration of that run.
 * Synchronises the device.  Returns 0, RIS_ERR_ARG, RIS_ERR_TIMEOUT (an MMA
 * completion wait timed out) or RIS_ERR_CUDA.
 */
int ris_debug_peak_probe(int kind, int reps, double* tflops, double* ms);

/*
 * Test hook: the number of device allocations (cudaMalloc, cudaMallocAsync)
 * the library has made since it was loaded, over all contexts, devices and
 * hooks.  Lets a test check that a call allocated nothing.
 */
long long ris_debug_alloc_count(void);

/* Message of the last error on this context ("" if none). */
const char* ris_last_error(const ris_ctx* ctx);

/* Free the context and everything it owns.  NULL is ignored. */
void ris_destroy(ris_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* RIS_H_ */
