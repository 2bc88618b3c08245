// TDDFT-ris engine: basis setup, metric factorisation, B tensors, Davidson
// excitation energies and the explicit nuclear derivatives of the ris pair
// energies.
//
// Notation (closed-shell singlet; i,j occupied, a,b virtual, P,Q auxiliary):
//   B^X_{pq,R} = sum_P (pq|P) (L_X^-T)_PR,  M_X = L_X L_X^T      (Eq. g_modified)
//   c^X_{pq,P} = sum_R B^X_{pq,R} (L_X^-1)_RP = sum_Q (pq|Q)(M_X^-1)_QP
//   (A X)_ia = (e_a - e_i) X_ia + 2 sum_R B^J_ia,R (B^J_R . X)
//              - c_x sum_R sum_jb B^K_ij,R X_jb B^K_ab,R        (Eq. A_matrix)
//   E_IJ = 1/2 [R_I (A+B) R_J + L_I (A-B) L_J], R = X+Y, L = X-Y  (Appendix A)
// The derivative of E_IJ at fixed C, eps and amplitudes follows the RI
// derivative formula closing Sec. 2.2:
//   dE_IJ/dxi = sum (mu nu|P)^xi Gamma_{mu nu,P} - sum_PQ (P|Q)^xi Omega_PQ
// with the three-index density Gamma of the pair, in the AO basis:
//   Coulomb (J set):  Gamma = 2 (D_I c_J + D_J c_I),  D_s = C_o R_s C_v^T,
//                     c_s = M_J^-1 (T^J . D_s),     Omega = 2 c_I c_J^T
//   exchange (K set), for each (U,V) in {(R_I,R_J),(L_I,L_J)} with weight
//   -c_x/2:  Gamma += C_o G^oo_P C_o^T + (U C_v^T)^T c^oo_P (V C_v^T),
//            G^oo_P = U c^vv_P V^T,  Omega += sum_ij c^oo_ij,P G^oo_ij,Q
//   and, for RPA, the (ib|ja) term with weights -c_x/2 (R,R) and +c_x/2 (L,L):
//            Gamma += C_o (U c^ov_P^T V + V c^ov_P^T U) C_v^T,
//            Omega += sum_ib c^ov_ib,P (U c^ov_Q^T V)_ib.
// The bra derivative tensor D^x_{mu nu,P} = (d_x mu nu|P) is contracted with
// the symmetrised Gamma; the auxiliary-centre and metric derivatives follow
// from translational invariance.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <set>

#include "engine.cuh"
#include "gemm_ff.cuh"

namespace ris {

thread_local MemTrack* t_track = nullptr;

void* dev_alloc(size_t bytes, cudaStream_t st, MemTrack** owner) {
  void* p = nullptr;
  ++g_allocs;
  cudaError_t e = cudaMallocAsync(&p, bytes, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error{RIS_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed"};
  }
  *owner = t_track;
  if (t_track) t_track->add((long long)bytes);
  return p;
}
void dev_free(void* p, size_t bytes, cudaStream_t st, MemTrack* owner) {
  cudaFreeAsync(p, st);
  if (owner) owner->cur -= (long long)bytes;
}

void ensure_smem_attr(const void* func, int bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  RIS_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({func, dev})) return;
  RIS_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.insert({func, dev});
}

void DBuf::ensure(size_t count, cudaStream_t s) {
  if (p && count <= n) return;
  release();
  if (count == 0) count = 1;
  st = s;
  p = (double*)dev_alloc(count * sizeof(double), st, &tr);
  n = count;
}
void DBuf::release() {
  if (p) dev_free(p, n * sizeof(double), st, tr);
  p = nullptr;
  n = 0;
}

void FBuf::ensure(size_t count, cudaStream_t s) {
  if (p && count <= n) return;
  release();
  if (count == 0) count = 1;
  st = s;
  p = (float*)dev_alloc(count * sizeof(float), st, &tr);
  n = count;
  RIS_CUDA(cudaMemsetAsync(p, 0, count * sizeof(float), st));
}
void FBuf::release() {
  if (p) dev_free(p, n * sizeof(float), st, tr);
  p = nullptr;
  n = 0;
}

static void free_shells(ShellSet& s, cudaStream_t st) {
  int** ip[] = {&s.atom, &s.l, &s.off, &s.jmap, &s.kmap, &s.fun_atom, &s.d_by_l[0], &s.d_by_l[1],
                &s.d_by_l[2]};
  for (auto q : ip)
    if (*q) {
      cudaFreeAsync(*q, st);
      *q = nullptr;
    }
  double** dp[] = {&s.ex, &s.nbase};
  for (auto q : dp)
    if (*q) {
      cudaFreeAsync(*q, st);
      *q = nullptr;
    }
}

void Engine::trim() {
  join_D();
  free_shells(ao, st);
  free_shells(aux, st);
  free_pairs(pl, st);
  if (d_jU) cudaFreeAsync(d_jU, st);
  if (d_kU) cudaFreeAsync(d_kU, st);
  if (d_kJ) cudaFreeAsync(d_kJ, st);
  d_jU = d_kU = d_kJ = nullptr;
  DBuf* dbs[] = {&xyz, &TJ, &TK, &MU, &dMU, &LJinv, &LKinv, &D, &C, &eps, &de, &BJ, &BKoo,
                 &BKvvD, &BKovR, &cKovP, &cKoo, &cKvv, &cKov, &cKooP, &omega, &X, &Y,
                 &w1, &w2, &w3, &w4, &w5, &w6, &w7, &w8};
  for (DBuf* b : dbs) b->release();
  FBuf* fbs[] = {&BooH, &BooL, &BvvH, &BvvL, &XtH, &XtL, &YH, &YL, &cvvH, &cvvL,
                 &cooH, &cooL, &CoH, &CoL, &CvH, &CvL, &Df};
  for (FBuf* b : fbs) b->release();
  aoPtr.release();
  aoList.release();
  axPtr.release();
  axList.release();
  nbPtr.release();
  nbCol.release();
  pOff.release();
  fpMu.release();
  fpNu.release();
  BJao.release();
  BKao.release();
  for (ShellSet& b : auxBlk) free_shells(b, st);
  auxBlk.clear();
  blkU0.clear();
  blkW.clear();
  blkWK.clear();
  streamed = false;
  have_D = false;
  stage = 0;
  nstates = 0;
  mem.peak = mem.cur;
}

Engine::~Engine() {
  trim();
  if (d_info) cudaFreeAsync(d_info, st);
  if (d_tcerr) cudaFreeAsync(d_tcerr, st);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (st) cudaStreamSynchronize(st);
  if (st2) cudaStreamSynchronize(st2);
  if (evA) cudaEventDestroy(evA);
  if (evD) cudaEventDestroy(evD);
}

template <class T>
static T* upload(const std::vector<T>& v, cudaStream_t st) {
  T* d = nullptr;
  RIS_ALLOC(cudaMallocAsync((void**)&d, sizeof(T) * std::max<size_t>(v.size(), 1), st));
  if (!v.empty())
    RIS_CUDA(cudaMemcpyAsync(d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
  return d;
}

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copy n doubles from a user pointer (host or device) into device memory.
static void copy_in(double* dst, const double* src, size_t n, cudaStream_t st) {
  RIS_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double),
                           is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           st));
}
// Copy n doubles from a user pointer (host or device) into host memory;
// a device source is read on the context's stream (no device-wide sync).
void copy_to_host(double* dst, const double* src, size_t n, cudaStream_t st) {
  if (is_device_ptr(src)) {
    RIS_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    RIS_CUDA(cudaStreamSynchronize(st));
  } else {
    memcpy(dst, src, n * sizeof(double));
  }
}
static void copy_out(double* dst, const double* src, size_t n, cudaStream_t st) {
  RIS_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double),
                           is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           st));
}

static void make_shells(ShellSet& s, const std::vector<int>& atom, const std::vector<int>& l,
                        const std::vector<double>& ex, const std::vector<int>* jmap,
                        const std::vector<int>* kmap, cudaStream_t st) {
  free_shells(s, st);
  s.n = (int)atom.size();
  s.h_atom = atom;
  s.h_l = l;
  s.h_ex = ex;
  s.h_off.assign(s.n, 0);
  std::vector<double> nb(s.n);
  std::vector<int> fa;
  int o = 0;
  for (int i = 0; i < s.n; i++) {
    s.h_off[i] = o;
    o += ncart(l[i]);
    for (int c = 0; c < ncart(l[i]); c++) fa.push_back(atom[i]);
    nb[i] = pow(2.0 * ex[i] / M_PI, 0.75) * pow(4.0 * ex[i], 0.5 * l[i]);
  }
  s.nfun = o;
  s.atom = upload(atom, st);
  s.l = upload(l, st);
  s.off = upload(s.h_off, st);
  s.ex = upload(ex, st);
  s.nbase = upload(nb, st);
  s.fun_atom = upload(fa, st);
  if (jmap) {
    s.h_jmap = *jmap;
    s.jmap = upload(*jmap, st);
  }
  if (kmap) {
    s.h_kmap = *kmap;
    s.kmap = upload(*kmap, st);
  }
  for (int L = 0; L <= kMaxLAux; L++) {
    s.by_l[L].clear();
    for (int i = 0; i < s.n; i++)
      if (l[i] == L) s.by_l[L].push_back(i);
    s.d_by_l[L] = upload(s.by_l[L], st);
  }
}

// ------------------------------------------------------------------ small kernels
__global__ void k_gather_sq(const double* __restrict__ src, int lds, const int* __restrict__ map,
                            int n, double* __restrict__ dst) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int i = t / n, j = t % n;
  dst[t] = src[(size_t)map[i] * lds + map[j]];
}

// dst[r][c] = src[r'][map[c]] (rows of length lds), c < nc, with r' = r, or,
// when n1 > 0, r = (i, j) -> r' = (j, i) for i < n0, j < n1 (row blocks
// transposed).
__global__ void k_gather_cols(const double* __restrict__ src, long long rows, int lds,
                              const int* __restrict__ map, int nc, double* __restrict__ dst, int n1,
                              int n0) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * nc) return;
  long long r = t / nc;
  const int c = (int)(t % nc);
  if (n1 > 0) r = (r % n1) * n0 + r / n1;
  dst[t] = src[(size_t)r * lds + map[c]];
}

__global__ void k_orb_diff(const double* __restrict__ eps, int nocc, int nvir, double* __restrict__ de) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nocc * nvir) return;
  de[t] = eps[nocc + t % nvir] - eps[t / nvir];
}

// out[b][R][a] = in[b][a][R]  (per b: transpose of an nvir x nR block)
__global__ void k_transpose_last2(const double* __restrict__ in, int nb, int na, int nr,
                                  double* __restrict__ out) {
  __shared__ double tile[32][33];
  const int b = blockIdx.z;
  const int a0 = blockIdx.x * 32, r0 = blockIdx.y * 32;  // the long index on grid.x
  const double* src = in + (size_t)b * na * nr;
  double* dst = out + (size_t)b * na * nr;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int a = a0 + k, r = r0 + threadIdx.x;
    tile[k][threadIdx.x] = (a < na && r < nr) ? src[(size_t)a * nr + r] : 0.0;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int r = r0 + k, a = a0 + threadIdx.x;
    if (r < nr && a < na) dst[(size_t)r * na + a] = tile[threadIdx.x][k];
  }
}
static void transpose_last2(const double* in, int nb, int na, int nr, double* out, cudaStream_t st) {
  RIS_REQUIRE(cdiv(nr, 32) <= 65535 && nb <= 65535, RIS_ERR_ARG, "transpose: shape too large");
  dim3 g(cdiv(na, 32), cdiv(nr, 32), nb);
  k_transpose_last2<<<g, dim3(32, 8), 0, st>>>(in, nb, na, nr, out);
  RIS_CHECK_LAUNCH();
}

// dst[r][c0 + c] = src[r][c] for c < ncol (FP32, row strides lds / ldd)
__global__ void k_copy_cols(const float* __restrict__ src, int lds, float* __restrict__ dst, int ldd,
                            int c0, int nrow, int ncol, long long dbatch) {
  // batch blockIdx.y: dst + blockIdx.y * dbatch (the same src for every batch)
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nrow * ncol) return;
  const int r = (int)(t / ncol), c = (int)(t % ncol);
  dst[(size_t)blockIdx.y * dbatch + (size_t)r * ldd + c0 + c] = src[(size_t)r * lds + c];
}

// out[c][a][b] = in[a][b][c]
__global__ void k_permute120(const double* __restrict__ in, int na, int nb, int nc,
                             double* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)na * nb * nc) return;
  const int c = (int)(t % nc);
  const long long ab = t / nc;
  const int b = (int)(ab % nb), a = (int)(ab / nb);
  out[((size_t)c * na + a) * nb + b] = in[t];
}

// out[b][a][c] = in[a][b][c]
__global__ void k_permute021(const double* __restrict__ in, int na, int nb, int nc,
                             double* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)na * nb * nc) return;
  const int c = (int)(t % nc);
  const long long ab = t / nc;
  const int b = (int)(ab % nb), a = (int)(ab / nb);
  out[((size_t)b * na + a) * nc + c] = in[t];
}

__global__ void k_add_diag(const double* __restrict__ de, const double* __restrict__ X, long long nov,
                           int nvec, double* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nov * nvec) return;
  out[t] += de[t % nov] * X[t];
}

// indices of the k smallest de (ties: smaller index first), one CTA
// Order-preserving integer key of a double (sign-magnitude to offset binary),
// so that the selection below compares integers, not FP64 values.
__device__ __forceinline__ unsigned long long dkey(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// idx[0..k) = indices of the k smallest de (ties by index), one block.
__global__ void __launch_bounds__(1024) k_lowest(const double* __restrict__ de, int n, int k,
                                                 int* __restrict__ idx) {
  __shared__ unsigned long long bv[32];
  __shared__ int bi[32];
  __shared__ unsigned long long lastv;
  __shared__ int lasti;
  if (threadIdx.x == 0) {
    lastv = 0ull;
    lasti = -1;
  }
  __syncthreads();
  for (int r = 0; r < k; r++) {
    unsigned long long best = ~0ull;
    int besti = 0x7fffffff;
    const unsigned long long lv = lastv;
    const int li = lasti;
    for (int i = threadIdx.x; i < n; i += 1024) {
      const unsigned long long v = dkey(de[i]);
      const bool after = (v > lv) || (v == lv && i > li);
      if (after && (v < best || (v == best && i < besti))) {
        best = v;
        besti = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, besti, o);
      if (ov < best || (ov == best && oi < besti)) {
        best = ov;
        besti = oi;
      }
    }
    if ((threadIdx.x & 31) == 0) {
      bv[threadIdx.x >> 5] = best;
      bi[threadIdx.x >> 5] = besti;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      best = bv[threadIdx.x];
      besti = bi[threadIdx.x];
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, besti, o);
        if (ov < best || (ov == best && oi < besti)) {
          best = ov;
          besti = oi;
        }
      }
      if (threadIdx.x == 0) {
        idx[r] = besti;
        lastv = best;
        lasti = besti;
      }
    }
    __syncthreads();
  }
}

__global__ void k_unit_rows(const int* __restrict__ idx, int k, long long n, double* __restrict__ V) {
  const int r = blockIdx.x;
  if (r >= k) return;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) V[(size_t)r * n + i] = (i == idx[r]) ? 1.0 : 0.0;
}

// R[k] = AX[k] - w[k] X[k]
__global__ void k_residual(const double* __restrict__ AX, const double* __restrict__ X,
                           const double* __restrict__ w, long long n, int ns, double* __restrict__ R) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ns) return;
  R[t] = AX[t] - w[t / n] * X[t];
}

// T[j] = R[u_j] / (de - w[u_j]), |denominator| floored at 1e-8
__global__ void k_precond(const double* __restrict__ R, const double* __restrict__ de,
                          const double* __restrict__ w, const int* __restrict__ u, long long n, int nt,
                          double* __restrict__ T) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nt) return;
  const int j = (int)(t / n);
  const long long i = t % n;
  const int s = u[j];
  double den = de[i] - w[s];
  if (fabs(den) < 1e-8) den = den < 0 ? -1e-8 : 1e-8;
  T[t] = R[(size_t)s * n + i] / den;
}

// X[a][b][R] and X[b][a][R] both set to their mean (a < b)
__global__ void k_sym_pairs(double* __restrict__ X, int v, int nR) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)v * v * nR) return;
  const int R = (int)(t % nR);
  const long long ab = t / nR;
  const int a = (int)(ab / v), b = (int)(ab % v);
  if (a >= b) return;
  double* p = X + ((size_t)a * v + b) * nR + R;
  double* q = X + ((size_t)b * v + a) * nR + R;
  const double m = 0.5 * (*p + *q);
  *p = m;
  *q = m;
}

// Shift of the Coulomb-exact preconditioner: this far below the smallest
// orbital-energy difference (Hartree), so that D - s stays positive.
constexpr double kPrecondGap = 2e-3;

// out[0] = min(x[0..n)); one block
__global__ void __launch_bounds__(1024) k_min(const double* __restrict__ x, long long n,
                                              double* __restrict__ out) {
  __shared__ double red[32];
  double m = 1e308;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) m = fmin(m, x[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 1e308;
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) out[0] = m;
  }
}

// dinv = 1 / (de - s), s = min(de) - gap;  W[i][R] = dinv[i] BJ[i][R]
// rows r0 .. r0 + nr - 1: dinv[i] = 1 / (de[i] - s), W[i - r0][P] = dinv[i] B^J[i][P]
__global__ void k_precond_setup(const double* __restrict__ de, const double* __restrict__ dmin,
                                long long r0, long long nr, double gap,
                                const double* __restrict__ BJ, int nJ, double* __restrict__ dinv,
                                double* __restrict__ W) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nr * nJ) return;
  const long long i = r0 + t / nJ;
  const double d = 1.0 / (de[i] - (dmin[0] - gap));
  W[t] = d * BJ[(size_t)r0 * nJ + t];
  if (t % nJ == 0) dinv[i] = d;
}

__global__ void k_add_identity(double* __restrict__ A, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) A[(size_t)i * n + i] += 1.0;
}

// T[j] = R[u_j] * dinv   (u null: row j)
__global__ void k_precond_scale(const double* __restrict__ R, const double* __restrict__ dinv,
                                const int* __restrict__ u, long long n, int nt, double* __restrict__ T) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nt) return;
  const long long i = t % n;
  const int row = u ? u[t / n] : (int)(t / n);
  T[t] = R[(size_t)row * n + i] * dinv[i];
}

// T -= f dinv * P (rows of length n)
__global__ void k_precond_update(double* __restrict__ T, const double* __restrict__ P,
                                 const double* __restrict__ dinv, long long n, int nt, double f) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nt) return;
  T[t] -= f * dinv[t % n] * P[t];
}

// X[r] /= sqrt(nrm2[r]) (rows of zero norm zeroed); 256 threads per block,
// each block forms the reciprocal norms of the rows it touches once (an FP64
// square root and division per element would load the narrow FP64 pipe).
__global__ void __launch_bounds__(256) k_scale_rows(double* __restrict__ X, long long n, int nrow,
                                                    const double* __restrict__ nrm2) {
  __shared__ double inv[256];
  const long long t0 = (long long)blockIdx.x * 256;
  const long long r0 = t0 / n;
  const long long r1 = min((long long)nrow - 1, (t0 + 255) / n);
  if ((long long)threadIdx.x <= r1 - r0) {
    const double s = nrm2[r0 + threadIdx.x];
    inv[threadIdx.x] = s > 0 ? 1.0 / sqrt(s) : 0.0;
  }
  __syncthreads();
  const long long t = t0 + threadIdx.x;
  if (t >= n * nrow) return;
  X[t] *= inv[t / n - r0];
}

// Cholesky of the Gram matrix G (nt x nt, unit diagonal expected) with
// dropping of (near-)dependent rows; P[i][c] such that the kept rows
// Tnew_i = sum_c P[i][c] T_c are orthonormal.  *nkeep = number kept.
// One warp: right-looking factorisation G = R^T R over the pivots in order
// (a pivot whose remaining diagonal is not above drop * G_jj is skipped and
// updates nothing), lanes over the columns of each update; then P = R^-T
// restricted to the kept pivots, lane q solving R^T y = e_q.
__global__ void __launch_bounds__(32) k_cholqr_small(const double* G, int nt, double drop,
                                                     double* P, int* nkeep, double* pivmin) {
  extern __shared__ double sh[];
  double* A = sh;            // working copy, upper triangle updated
  double* R = A + nt * nt;   // row j: row of R for kept pivot j
  double* Ps = R + nt * nt;
  double* rinv = Ps + nt * nt;
  int* keep = (int*)(rinv + nt);
  const int lane = threadIdx.x;
  for (int i = lane; i < nt * nt; i += 32) {
    A[i] = G[i];
    R[i] = 0.0;
    Ps[i] = 0.0;
  }
  __syncwarp();
  int r = 0;
  double dmin = 1.0;  // smallest kept pivot relative to its diagonal
  for (int j = 0; j < nt; j++) {
    const double d = A[j * nt + j];
    if (!(d > drop * G[j * nt + j] && d > 0)) continue;  // warp-uniform
    dmin = fmin(dmin, d / G[j * nt + j]);
    const double rjj = sqrt(d), ri = 1.0 / rjj;
    for (int l = j + 1 + lane; l < nt; l += 32) R[j * nt + l] = A[j * nt + l] * ri;
    if (lane == 0) {
      R[j * nt + j] = rjj;
      rinv[r] = ri;
      keep[r] = j;
    }
    __syncwarp();
    for (int l2 = j + 1 + lane; l2 < nt; l2 += 32) {
      const double b = R[j * nt + l2];
      for (int l = j + 1; l <= l2; l++) A[l * nt + l2] -= R[j * nt + l] * b;
    }
    __syncwarp();
    r++;
  }
  // column keep[q] of P: y_s = (delta_sq - sum_{q <= s2 < s} R[keep s2][keep s] y_s2) / R_ss
  for (int q = lane; q < r; q += 32) {
    const int cq = keep[q];
    for (int s = q; s < r; s++) {
      double acc = s == q ? 1.0 : 0.0;
      const int ks = keep[s];
      for (int s2 = q; s2 < s; s2++) acc -= R[keep[s2] * nt + ks] * Ps[s2 * nt + cq];
      Ps[s * nt + cq] = acc * rinv[s];
    }
  }
  __syncwarp();
  if (lane == 0) {
    *nkeep = r;
    if (pivmin) *pivmin = dmin;
  }
  for (int i = lane; i < nt * nt; i += 32) P[i] = Ps[i];
}

// FP64 GEMM, or the double-FP32 one (gemm_ff.cu) when ff is set and the
// shape is one of its skinny forms.
static void gemm_sub(bool ff, bool ta, bool tb, int m, int n, int k, double alpha, const double* A,
                     int lda, const double* B, int ldb, double beta, double* C, int ldc,
                     cudaStream_t st) {
  if (!(ff && ffgemm(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, st)))
    dgemm(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, st);
}

static void cholqr_small(const double* G, int nt, double drop, double* P, int* nkeep,
                         cudaStream_t st, double* pivmin = nullptr) {
  RIS_REQUIRE(nt >= 1 && nt <= 64, RIS_ERR_ARG, "cholqr_small: block of 1..64 vectors");
  const size_t smem = (3 * (size_t)nt * nt + nt) * sizeof(double) + nt * sizeof(int);
  ensure_smem_attr((const void*)k_cholqr_small, (int)((3 * 64 * 64 + 64) * sizeof(double) + 64 * sizeof(int)));
  k_cholqr_small<<<1, 32, smem, st>>>(G, nt, drop, P, nkeep, pivmin);
  RIS_CHECK_LAUNCH();
}

__global__ void k_diag_set(double* __restrict__ H, int ld, int m, const double* __restrict__ w) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * m) return;
  const int i = t / m, j = t % m;
  H[(size_t)i * ld + j] = i == j ? w[i] : 0.0;
}

__global__ void k_mirror(double* __restrict__ H, int ld, int m0, int m1) {
  // for i in [m0, m1), j in [0, m0): H[j][i] = H[i][j]
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (m1 - m0) * m0) return;
  const int i = m0 + t / m0, j = t % m0;
  H[(size_t)j * ld + i] = H[(size_t)i * ld + j];
}

// Sign of each row so that its largest-magnitude element is positive
// (ties: smallest index); the same sign is applied to Y when given.
// |x| compared as the integer bit pattern of the magnitude (same order for
// non-negative doubles) so that the scan stays off the FP64 pipe.
__global__ void k_phase(double* __restrict__ X, double* __restrict__ Y, long long n) {
  __shared__ unsigned long long bv[32];
  __shared__ long long bi[32];
  __shared__ double sgn;
  double* x = X + (size_t)blockIdx.x * n;
  unsigned long long best = 0ull;
  long long besti = 0x7fffffffffffffffLL;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const unsigned long long v = (unsigned long long)__double_as_longlong(x[i]) & 0x7fffffffffffffffull;
    if (v > best || (v == best && i < besti)) {
      best = v;
      besti = i;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ov = __shfl_xor_sync(0xffffffffu, best, o);
    const long long oi = __shfl_xor_sync(0xffffffffu, besti, o);
    if (ov > best || (ov == best && oi < besti)) {
      best = ov;
      besti = oi;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    bv[threadIdx.x >> 5] = best;
    bi[threadIdx.x >> 5] = besti;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++)
      if (bv[w] > bv[0] || (bv[w] == bv[0] && bi[w] < bi[0])) {
        bv[0] = bv[w];
        bi[0] = bi[w];
      }
    sgn = x[bi[0]] < 0 ? -1.0 : 1.0;
  }
  __syncthreads();
  if (sgn < 0) {
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
      x[i] = -x[i];
      if (Y) Y[(size_t)blockIdx.x * n + i] = -Y[(size_t)blockIdx.x * n + i];
    }
  }
}

__global__ void k_axpby(long long n, double a, const double* __restrict__ x, double b,
                        const double* __restrict__ y, double* __restrict__ z) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) z[t] = a * x[t] + (y ? b * y[t] : 0.0);
}
static void axpby(long long n, double a, const double* x, double b, const double* y, double* z,
                  cudaStream_t st) {
  if (n <= 0) return;
  k_axpby<<<cdiv(n, 256), 256, 0, st>>>(n, a, x, b, y, z);
  RIS_CHECK_LAUNCH();
}

// Gamma[mu][nu][jU[P]] += f (DI[mu][nu] cJ[P] + DJ[mu][nu] cI[P])
// Symmetrise n x n matrices in place: X = (X + X^T) / 2, nb of them.
__global__ void k_symmetrize_sq(double* __restrict__ X, int n, int nb) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)nb * n * n) return;
  const int b = (int)(t / ((long long)n * n));
  const long long ij = t % ((long long)n * n);
  const int i = (int)(ij / n), j = (int)(ij % n);
  if (i >= j) return;
  double* M = X + (size_t)b * n * n;
  const double m = 0.5 * (M[(size_t)i * n + j] + M[(size_t)j * n + i]);
  M[(size_t)i * n + j] = m;
  M[(size_t)j * n + i] = m;
}

// cU[s][jU[Q]] = cJ[s][Q] (union index), zero elsewhere (cU zeroed by the caller)
__global__ void k_expand_cJ(const double* __restrict__ cJ, const int* __restrict__ jU, int ns,
                            int nJ, int nU, double* __restrict__ cU) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ns * nJ) return;
  const int s = t / nJ, Q = t % nJ;
  cU[(size_t)s * nU + jU[Q]] = cJ[t];
}

// Omega[jU[P]][jU[Q]] = f cI[P] cJ[Q]   (whole matrix zeroed first by caller)
__global__ void k_omega_J(const double* __restrict__ cI, const double* __restrict__ cJ,
                          const int* __restrict__ jU, int nJ, int nU, double f, double* __restrict__ O) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nJ * nJ) return;
  const int P = t / nJ, Q = t % nJ;
  O[(size_t)jU[P] * nU + jU[Q]] += f * cI[P] * cJ[Q];
}

// W_V[nu][k] = C_o[nu][k] (k < o), Q[k-o][nu] (k >= o)
__global__ void k_build_W(const double* __restrict__ C, int nmo, const double* __restrict__ Q,
                          int nao, int nocc, double* __restrict__ W) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nao * 2 * nocc) return;
  const int nu = t / (2 * nocc), k = t % (2 * nocc);
  W[t] = k < nocc ? C[(size_t)nu * nmo + k] : Q[(size_t)(k - nocc) * nao + nu];
}

constexpr int kCBatch = 8;  // states (or pairs) sharing one pass over the derivative integrals

// The contractions below run one thread per (mu, P, slice of nu): the sum
// over nu runs over mu's screened partners only (the derivative integrals
// vanish elsewhere; CSR lists nbPtr / nbCol) and is cut into nslice slices so
// that enough warps are in flight, each slice writes its partial sums and
// k_sum_slices adds them in a fixed order.
// With T = float (mixed precision: derivative integrals stored in FP32) the
// products and runs of kChunk terms are summed in FP32 and the runs in FP64;
// with T = double everything is FP64.
constexpr int kChunk = 32;

__host__ __device__ inline void slice_range(int nao, int nslice, int s, int& lo, int& hi) {
  lo = (int)((long long)nao * s / nslice);
  hi = (int)((long long)nao * (s + 1) / nslice);
}

// State densities regrouped for the contraction: DRt[batch][mu][nu][b] =
// DR_{8 batch + b}[mu][nu] (zero past the last state), so that a partner's
// eight weights are two (FP32) or four (FP64) vector loads.
template <class T>
__global__ void k_states_t(const double* __restrict__ DR, int nsu, int nao, T* __restrict__ out) {
  const long long nn2 = (long long)nao * nao;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nn2) return;
  const int batch = blockIdx.y;
  T v[kCBatch];
#pragma unroll
  for (int b = 0; b < kCBatch; b++) {
    const int s = batch * kCBatch + b;
    v[b] = s < nsu ? (T)DR[(size_t)s * nn2 + t] : (T)0;
  }
  T* o = out + ((size_t)batch * nn2 + t) * kCBatch;
#pragma unroll
  for (int b = 0; b < kCBatch; b++) o[b] = v[b];
}

__device__ __forceinline__ void load_w8(const float* p, float (&w)[kCBatch]) {
  const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
  w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w; w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
}
__device__ __forceinline__ void load_w8(const double* p, double (&w)[kCBatch]) {
#pragma unroll
  for (int h = 0; h < 4; h++) {
    const double2 a = *reinterpret_cast<const double2*>(p + 2 * h);
    w[2 * h] = a.x;
    w[2 * h + 1] = a.y;
  }
}

// Coulomb part, per state (the pair densities are linear in the per-state
// transition densities): part[slice][b][x][mu][P] = sum_{nu in slice}
// D[x][mu][nu][P] DRt[mu][nu][b], b < ns <= kCBatch, DRt the batch's
// symmetrised state densities regrouped by k_states_t.
template <class T>
__global__ void __launch_bounds__(128) k_contract_states(const T* __restrict__ D,
                                                         const T* __restrict__ DRt, int ns,
                                                         int nao, int nU, int nslice,
                                                         const int* __restrict__ nbPtr,
                                                         const int* __restrict__ nbCol,
                                                         double* __restrict__ part) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nao * nU) return;
  const int mu = (int)(idx / nU), P = (int)(idx % nU);
  int q0, q1;  // this slice of mu's screened partners nu
  slice_range(nbPtr[mu + 1] - nbPtr[mu], nslice, blockIdx.y, q0, q1);
  q0 += nbPtr[mu];
  q1 += nbPtr[mu];
  const size_t nn2 = (size_t)nao * nao;
  const size_t plane = nn2 * nU;
  double y[kCBatch][3];
  T c[kCBatch][3];
#pragma unroll
  for (int b = 0; b < kCBatch; b++)
#pragma unroll
    for (int x = 0; x < 3; x++) y[b][x] = 0.0, c[b][x] = (T)0;
  const T* dr = DRt + (size_t)mu * nao * kCBatch;
  // runs of kChunk partners: products summed in T, runs in FP64; the inner
  // loop is unrolled so that several partners' loads are in flight
  for (int qc = q0; qc < q1; qc += kChunk) {
    const int qe = min(qc + kChunk, q1);
#pragma unroll 4
    for (int q = qc; q < qe; q++) {
      const int nu = nbCol[q];
      const size_t a = ((size_t)mu * nao + nu) * nU + P;
      const T d0 = D[a], d1 = D[plane + a], d2 = D[2 * plane + a];
      T w[kCBatch];
      load_w8(dr + (size_t)nu * kCBatch, w);
#pragma unroll
      for (int b = 0; b < kCBatch; b++) {
        if (b >= ns) break;
        c[b][0] += d0 * w[b];
        c[b][1] += d1 * w[b];
        c[b][2] += d2 * w[b];
      }
    }
#pragma unroll
    for (int b = 0; b < kCBatch; b++)
#pragma unroll
      for (int x = 0; x < 3; x++) y[b][x] += (double)c[b][x], c[b][x] = (T)0;
  }
  double* ps = part + (size_t)blockIdx.y * ns * 3 * nao * nU;
#pragma unroll
  for (int b = 0; b < kCBatch; b++) {
    if (b >= ns) break;
#pragma unroll
    for (int x = 0; x < 3; x++) ps[(((size_t)b * 3 + x) * nao + mu) * nU + P] = y[b][x];
  }
}

// Exchange part, per pair of a batch (nb <= kCBatch), P < nK:
//   part[slice][g][x][mu][P] = sum_{nu in slice} D[x][mu][nu][P]
//                              (GK_g[mu][nu][P] + GK_g[nu][mu][P]) / 2
template <class T, class G>
__global__ void __launch_bounds__(128) k_contract_exchange(const T* __restrict__ D,
                                                           const G* __restrict__ GK, int nb,
                                                           int nao, int nU, int nK, int nslice,
                                                           const int* __restrict__ nbPtr,
                                                           const int* __restrict__ nbCol,
                                                           double* __restrict__ part) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nao * nK) return;
  const int mu = (int)(idx / nK), P = (int)(idx % nK);
  int q0, q1;  // this slice of mu's screened partners nu
  slice_range(nbPtr[mu + 1] - nbPtr[mu], nslice, blockIdx.y, q0, q1);
  q0 += nbPtr[mu];
  q1 += nbPtr[mu];
  const size_t nn2 = (size_t)nao * nao;
  const size_t plane = nn2 * nU;
  const size_t gk = nn2 * nK;
  double s[kCBatch][3];
  T c[kCBatch][3];
#pragma unroll
  for (int b = 0; b < kCBatch; b++)
#pragma unroll
    for (int x = 0; x < 3; x++) s[b][x] = 0.0, c[b][x] = (T)0;
  for (int qc = q0; qc < q1; qc += kChunk) {
    const int qe = min(qc + kChunk, q1);
#pragma unroll 2
    for (int q = qc; q < qe; q++) {
      const int nu = nbCol[q];
      const size_t mn = (size_t)mu * nao + nu;
      const size_t a = mn * nU + P;
      const T d0 = D[a], d1 = D[plane + a], d2 = D[2 * plane + a];
      const size_t k1 = mn * nK + P, k2 = ((size_t)nu * nao + mu) * nK + P;
#pragma unroll
      for (int b = 0; b < kCBatch; b++) {
        if (b >= nb) break;
        const T g = (T)0.5 * ((T)GK[b * gk + k1] + (T)GK[b * gk + k2]);
        c[b][0] += d0 * g;
        c[b][1] += d1 * g;
        c[b][2] += d2 * g;
      }
    }
#pragma unroll
    for (int b = 0; b < kCBatch; b++)
#pragma unroll
      for (int x = 0; x < 3; x++) s[b][x] += (double)c[b][x], c[b][x] = (T)0;
  }
  double* ps = part + (size_t)blockIdx.y * nb * 3 * nao * nK;
#pragma unroll
  for (int b = 0; b < kCBatch; b++) {
    if (b >= nb) break;
#pragma unroll
    for (int x = 0; x < 3; x++) ps[(((size_t)b * 3 + x) * nao + mu) * nK + P] = s[b][x];
  }
}

// out[i] = sum_s part[s][i], i < n (fixed order)
__global__ void k_sum_slices(const double* __restrict__ part, int nslice, long long n,
                             double* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int sl = 0; sl < nslice; sl++) acc += part[(size_t)sl * n + i];
  out[i] = acc;
}

// slices of the nu sum so that about eight blocks per SM are in flight
static int pick_slices(long long threads, int partners) {
  const int base = cdiv(threads, 128);
  return std::max(1, std::min({cdiv(8 * 152, base), partners / 16, 64}));
}

// W_g[x][mu][P] of pair g = (I, J): exchange part plus the Coulomb part
// 2 (cU_J[P] Y_I[x][mu][P] + cU_I[P] Y_J[x][mu][P]).
__device__ __forceinline__ double pair_w(const double* WKg, const double* YI, const double* YJ,
                                         const double* cI, const double* cJ, int x, int mu, int P,
                                         int nao, int nU, int nK) {
  const size_t y = ((size_t)x * nao + mu) * nU + P;
  double w = 2.0 * (cJ[P] * YI[y] + cI[P] * YJ[y]);
  if (P < nK) w += WKg[((size_t)x * nao + mu) * nK + P];
  return w;
}

// grad[g][A][x] = 2 sum_{mu in A, P} W_g - 2 sum_{P in A, mu} W_g
//                 - sum_{P in A, Q} (O[P][Q] + O[Q][P]) dM[x][P][Q]
// (block (A, g); the functions of atom A from the CSR lists)
__global__ void __launch_bounds__(128) k_grad_reduce_pairs(
    const double* __restrict__ WK, const double* __restrict__ Y, const double* __restrict__ cU,
    const int* __restrict__ pst, const double* __restrict__ O, const double* __restrict__ dM,
    const int* __restrict__ aoPtr, const int* __restrict__ aoList, const int* __restrict__ axPtr,
    const int* __restrict__ axList, int nao, int nU, int nK, int natm,
    double* __restrict__ grad) {
  __shared__ double red[3][128];
  const int A = blockIdx.x, g = blockIdx.y;
  const int sI = pst[2 * g], sJ = pst[2 * g + 1];
  const double* WKg = WK + (size_t)g * 3 * nao * nK;
  const double* YI = Y + (size_t)sI * 3 * nao * nU;
  const double* YJ = Y + (size_t)sJ * 3 * nao * nU;
  const double* cI = cU + (size_t)sI * nU;
  const double* cJ = cU + (size_t)sJ * nU;
  const double* Og = O + (size_t)g * nU * nU;
  double s[3] = {0.0, 0.0, 0.0};
  const int a0 = aoPtr[A], na = aoPtr[A + 1] - a0;
  for (long long t = threadIdx.x; t < (long long)na * nU; t += 128) {
    const int mu = aoList[a0 + (int)(t / nU)], P = (int)(t % nU);
#pragma unroll
    for (int x = 0; x < 3; x++) s[x] += 2.0 * pair_w(WKg, YI, YJ, cI, cJ, x, mu, P, nao, nU, nK);
  }
  const int p0 = axPtr[A], np = axPtr[A + 1] - p0;
  for (long long t = threadIdx.x; t < (long long)np * nao; t += 128) {
    const int P = axList[p0 + (int)(t / nao)], mu = (int)(t % nao);
#pragma unroll
    for (int x = 0; x < 3; x++) s[x] -= 2.0 * pair_w(WKg, YI, YJ, cI, cJ, x, mu, P, nao, nU, nK);
  }
  for (long long t = threadIdx.x; t < (long long)np * nU; t += 128) {
    const int P = axList[p0 + (int)(t / nU)], Q = (int)(t % nU);
    const double o = Og[(size_t)P * nU + Q] + Og[(size_t)Q * nU + P];
#pragma unroll
    for (int x = 0; x < 3; x++) s[x] -= o * dM[((size_t)x * nU + P) * nU + Q];
  }
  for (int x = 0; x < 3; x++) red[x][threadIdx.x] = s[x];
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int x = 0; x < 3; x++) red[x][threadIdx.x] += red[x][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 3) grad[((size_t)g * natm + A) * 3 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void k_divide_pairs(double* __restrict__ out, const double* __restrict__ num,
                               const double* __restrict__ den, int npair, int per) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npair * per) return;
  out[t] = num[t] / den[t / per];
}

void divide_pairs(double* out, const double* num, const double* den, int npair, int per,
                  cudaStream_t st) {
  k_divide_pairs<<<cdiv((long long)npair * per, 256), 256, 0, st>>>(out, num, den, npair, per);
  RIS_CHECK_LAUNCH();
}

// out[j] = A_j . B_j (rows of length n), one block per row
__global__ void k_row_dots(const double* __restrict__ A, const double* __restrict__ B, long long n,
                           double* __restrict__ out) {
  __shared__ double red[8];
  const double* a = A + (size_t)blockIdx.x * n;
  const double* b = B + (size_t)blockIdx.x * n;
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += 256) s += a[i] * b[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; w++) t += red[w];
    out[blockIdx.x] = t;
  }
}

// CG update for row j with step a[j] = rz[j] / pq[j] (0 for frozen rows):
//   x_j += a p_j,  r_j -= a q_j
__global__ void k_cg_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                        const double* __restrict__ q, const double* __restrict__ rz,
                        const double* __restrict__ pq, const int* __restrict__ active, long long n,
                        int nr) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nr) return;
  const int j = (int)(t / n);
  if (!active[j]) return;
  const double a = rz[j] / pq[j];
  x[t] += a * p[t];
  r[t] -= a * q[t];
}

// p_j = z_j + (rz_new[j] / rz[j]) p_j for active rows
__global__ void k_cg_p(double* __restrict__ p, const double* __restrict__ z,
                       const double* __restrict__ rzn, const double* __restrict__ rz,
                       const int* __restrict__ active, long long n, int nr) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nr) return;
  const int j = (int)(t / n);
  if (!active[j]) return;
  p[t] = z[t] + (rzn[j] / rz[j]) * p[t];
}

// Phase of state blockIdx.x against the previous step: the overlap over the
// five largest |X_prev| determinants (ties by index); a negative overlap
// flips X (and Y) of the state.  sign[I] = +1 or -1.
__global__ void __launch_bounds__(256) k_phase_align(double* __restrict__ X, double* __restrict__ Y,
                                                     const double* __restrict__ Xp, long long n,
                                                     int* __restrict__ sign) {
  __shared__ unsigned long long bk[8];
  __shared__ long long bi[8];
  __shared__ long long top[5];
  __shared__ double ov;
  if (threadIdx.x < 5) top[threadIdx.x] = -1;
  __syncthreads();
  const int I = blockIdx.x;
  const double* xp = Xp + (size_t)I * n;
  double* x = X + (size_t)I * n;
  unsigned long long lastk = ~0ull;
  long long lasti = -1;
  for (int r = 0; r < 5; r++) {
    // largest |xp| strictly after (lastk, lasti) in the order (|x| desc, index asc)
    unsigned long long best = 0;
    long long besti = -1;
    for (long long i = threadIdx.x; i < n; i += 256) {
      const unsigned long long k = (unsigned long long)__double_as_longlong(fabs(xp[i]));
      const bool after = lasti < 0 || k < lastk || (k == lastk && i > lasti);
      if (after && (besti < 0 || k > best || (k == best && i < besti))) {
        best = k;
        besti = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ok = __shfl_xor_sync(0xffffffffu, best, o);
      const long long oi = __shfl_xor_sync(0xffffffffu, besti, o);
      if (oi >= 0 && (besti < 0 || ok > best || (ok == best && oi < besti))) {
        best = ok;
        besti = oi;
      }
    }
    if ((threadIdx.x & 31) == 0) {
      bk[threadIdx.x >> 5] = best;
      bi[threadIdx.x >> 5] = besti;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < 8; w++)
        if (bi[w] >= 0 && (bi[0] < 0 || bk[w] > bk[0] || (bk[w] == bk[0] && bi[w] < bi[0]))) {
          bk[0] = bk[w];
          bi[0] = bi[w];
        }
      top[r] = bi[0];
    }
    __syncthreads();
    lastk = bk[0];
    lasti = bi[0];
    __syncthreads();
    if (lasti < 0) break;  // fewer than five elements
  }
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int r = 0; r < 5; r++)
      if (top[r] >= 0) s += x[top[r]] * xp[top[r]];
    ov = s;
    sign[I] = s < 0.0 ? -1 : 1;
  }
  __syncthreads();
  if (ov < 0.0) {
    for (long long i = threadIdx.x; i < n; i += 256) x[i] = -x[i];
    if (Y)
      for (long long i = threadIdx.x; i < n; i += 256) Y[(size_t)I * n + i] = -Y[(size_t)I * n + i];
  }
}

// RPA operators from their parts: P = de Z + 4 J - cx (K1 + K2), M = de Z - cx (K1 - K2);
// on entry outP holds J.
__global__ void k_rpa_combine(const double* __restrict__ de, const double* __restrict__ Z,
                              const double* __restrict__ K1, const double* __restrict__ K2,
                              long long nov, int nvec, double cx, double* __restrict__ outP,
                              double* __restrict__ outM) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nov * nvec) return;
  const double dz = de[t % nov] * Z[t];
  outP[t] = dz + 4.0 * outP[t] - cx * (K1[t] + K2[t]);
  if (outM) outM[t] = dz - cx * (K1[t] - K2[t]);
}

// ------------------------------------------------------------------ setup
// nbPtr / nbCol: the screened partners nu of every AO function mu (both
// orders of each screened shell pair), by counting then filling; the order
// within a row is that of the pair list (deterministic).
void Engine::partners_from_host_pairs() {
  const int nf = ao.nfun;
  std::vector<int> ptr(nf + 1, 0);
  for (int ip = 0; ip < pl.npair; ip++) {
    const int sa = h_pa[ip], sb = h_pb[ip];
    const int na = ncart(ao.h_l[sa]), nb = ncart(ao.h_l[sb]);
    for (int ia = 0; ia < na; ia++) ptr[ao.h_off[sa] + ia + 1] += nb;
    if (sa != sb)
      for (int ib = 0; ib < nb; ib++) ptr[ao.h_off[sb] + ib + 1] += na;
  }
  for (int mu = 0; mu < nf; mu++) ptr[mu + 1] += ptr[mu];
  std::vector<int> col(std::max(ptr[nf], 1)), fill(ptr.begin(), ptr.end() - 1);
  for (int ip = 0; ip < pl.npair; ip++) {
    const int sa = h_pa[ip], sb = h_pb[ip];
    const int na = ncart(ao.h_l[sa]), nb = ncart(ao.h_l[sb]);
    for (int ia = 0; ia < na; ia++)
      for (int ib = 0; ib < nb; ib++) {
        const int mu = ao.h_off[sa] + ia, nu = ao.h_off[sb] + ib;
        col[fill[mu]++] = nu;
        if (sa != sb) col[fill[nu]++] = mu;
      }
  }
  nbAvg = std::max(1, ptr[nf] / std::max(nf, 1));
  nbPtr.ensure(nf + 1, st);
  nbCol.ensure(col.size(), st);
  // pageable host-to-device copies are staged before the call returns
  RIS_CUDA(cudaMemcpyAsync(nbPtr.p, ptr.data(), sizeof(int) * (nf + 1), cudaMemcpyHostToDevice, st));
  RIS_CUDA(cudaMemcpyAsync(nbCol.p, col.data(), sizeof(int) * col.size(), cudaMemcpyHostToDevice, st));
}

void Engine::build_aux(int natm_, const double* coords, int nshell, const ris_shell* aos, int nJs,
                       const ris_shell* auxJ, int nKs, const ris_shell* auxK) {
  RIS_REQUIRE(natm_ > 0 && nshell > 0 && nJs > 0 && nKs > 0, RIS_ERR_ARG, "empty input");
  RIS_REQUIRE(coords && aos && auxJ && auxK, RIS_ERR_ARG, "null pointer");
  std::vector<double> hxyz(3 * (size_t)natm_);
  copy_to_host(hxyz.data(), coords, 3 * (size_t)natm_, st);
  for (double v : hxyz) RIS_REQUIRE(std::isfinite(v), RIS_ERR_ARG, "non-finite coordinate");
  auto check = [&](const ris_shell* s, int n, int lmax, const char* what) {
    for (int i = 0; i < n; i++) {
      RIS_REQUIRE(s[i].atom >= 0 && s[i].atom < natm_, RIS_ERR_ARG,
                  std::string(what) + ": atom index out of range");
      RIS_REQUIRE(s[i].l >= 0 && s[i].l <= lmax, RIS_ERR_ARG,
                  std::string(what) + ": angular momentum out of range");
      RIS_REQUIRE(s[i].exponent > 0 && std::isfinite(s[i].exponent), RIS_ERR_ARG,
                  std::string(what) + ": bad exponent");
    }
  };
  check(aos, nshell, kMaxLAO, "AO shell");
  check(auxJ, nJs, kMaxLAux, "J auxiliary shell");
  check(auxK, nKs, kMaxLAux, "K auxiliary shell");
  join_D();  // a previous geometry's derivative integrals may still read the shells
  stage = 0;
  have_D = false;
  natm = natm_;
  xyz.ensure(3 * (size_t)natm, st);
  RIS_CUDA(cudaMemcpyAsync(xyz.p, hxyz.data(), sizeof(double) * 3 * natm, cudaMemcpyHostToDevice, st));
  // AO shells
  {
    std::vector<int> a(nshell), l(nshell);
    std::vector<double> e(nshell);
    for (int i = 0; i < nshell; i++) {
      a[i] = aos[i].atom;
      l[i] = aos[i].l;
      e[i] = aos[i].exponent;
    }
    make_shells(ao, a, l, e, nullptr, nullptr, st);
  }
  // union auxiliary set: K shells first, then J shells not already present
  {
    std::vector<int> a, l, jm, km;
    std::vector<double> e;
    std::vector<int> joff(nJs), koff(nKs);
    int o = 0;
    for (int i = 0; i < nJs; i++) {
      joff[i] = o;
      o += ncart(auxJ[i].l);
    }
    nJ = o;
    o = 0;
    for (int i = 0; i < nKs; i++) {
      koff[i] = o;
      o += ncart(auxK[i].l);
    }
    nK = o;
    auto same = [](const ris_shell& x, const ris_shell& y) {
      return x.atom == y.atom && x.l == y.l && x.exponent == y.exponent;
    };
    std::vector<bool> used(nJs, false);
    for (int i = 0; i < nKs; i++) {
      a.push_back(auxK[i].atom);
      l.push_back(auxK[i].l);
      e.push_back(auxK[i].exponent);
      km.push_back(koff[i]);
      int jj = -1;
      for (int j = 0; j < nJs; j++)
        if (!used[j] && same(auxJ[j], auxK[i])) {
          jj = j;
          break;
        }
      if (jj >= 0) used[jj] = true;
      jm.push_back(jj >= 0 ? joff[jj] : -1);
    }
    for (int j = 0; j < nJs; j++)
      if (!used[j]) {
        a.push_back(auxJ[j].atom);
        l.push_back(auxJ[j].l);
        e.push_back(auxJ[j].exponent);
        jm.push_back(joff[j]);
        km.push_back(-1);
      }
    make_shells(aux, a, l, e, &jm, &km, st);
    nU = aux.nfun;
    nKsh = nKs;
    // functions of each atom (CSR) for the per-atom gradient sums
    auto csr = [&](const ShellSet& sh, SBuf<int>& ptr, SBuf<int>& list) {
      std::vector<int> cnt(natm + 1, 0), lst;
      std::vector<std::vector<int>> per(natm);
      for (int i = 0; i < sh.n; i++)
        for (int c = 0; c < ncart(sh.h_l[i]); c++) per[sh.h_atom[i]].push_back(sh.h_off[i] + c);
      for (int A = 0; A < natm; A++) {
        cnt[A + 1] = cnt[A] + (int)per[A].size();
        lst.insert(lst.end(), per[A].begin(), per[A].end());
      }
      ptr.ensure(natm + 1, st);
      list.ensure(std::max<size_t>(lst.size(), 1), st);
      RIS_CUDA(cudaMemcpyAsync(ptr.p, cnt.data(), sizeof(int) * (natm + 1), cudaMemcpyHostToDevice, st));
      // pageable host-to-device copies are staged before the call returns
      RIS_CUDA(cudaMemcpyAsync(list.p, lst.data(), sizeof(int) * lst.size(), cudaMemcpyHostToDevice, st));
    };
    csr(ao, aoPtr, aoList);
    csr(aux, axPtr, axList);
    h_jU.assign(nJ, -1);
    h_kU.assign(nK, -1);
    for (int s = 0; s < aux.n; s++)
      for (int c = 0; c < ncart(l[s]); c++) {
        if (jm[s] >= 0) h_jU[jm[s] + c] = aux.h_off[s] + c;
        if (km[s] >= 0) h_kU[km[s] + c] = aux.h_off[s] + c;
      }
    if (d_jU) cudaFreeAsync(d_jU, st);
    if (d_kU) cudaFreeAsync(d_kU, st);
    if (d_kJ) cudaFreeAsync(d_kJ, st);
    d_jU = upload(h_jU, st);
    d_kU = upload(h_kU, st);
    // K fitting functions that are also J fitting functions (the minimal
    // K set of s functions inside the s+p J set): the K half transform is
    // then a column subset of the J one
    d_kJ = nullptr;
    {
      std::vector<int> uJ(nU, -1);
      for (int j = 0; j < nJ; j++) uJ[h_jU[j]] = j;
      h_kJ.assign(nK, -1);
      bool subset = true;
      for (int k = 0; k < nK; k++) {
        h_kJ[k] = uJ[h_kU[k]];
        subset = subset && h_kJ[k] >= 0;
      }
      if (subset) d_kJ = upload(h_kJ, st);
    }
  }
  // screened pair list; the estimate is scaled by the largest auxiliary
  // potential |V_P| <= N_P 2 pi / g (times g^-1/2 for p)
  double vmax = 0.0;
  for (int s = 0; s < aux.n; s++) {
    const double g = aux.h_ex[s];
    const double nb = pow(2.0 * g / M_PI, 0.75) * pow(4.0 * g, 0.5 * aux.h_l[s]);
    vmax = std::max(vmax, nb * 2.0 * M_PI / g * (aux.h_l[s] ? 1.0 / sqrt(g) : 1.0));
  }
  build_pairs(ao, xyz.p, opt.screen_thr / std::max(vmax, 1e-300), pl, nullptr, st);
  // the screened pairs go to pinned host memory on a copy stream, so that
  // each AO function's partner list is built on the host while the
  // integrals and the metric factors run on the device
  if (!st3) {  // high priority: its single-CTA metric factorisations run beside the integrals
    int lo = 0, hi = 0;
    RIS_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    RIS_CUDA(cudaStreamCreateWithPriority(&st3, cudaStreamNonBlocking, hi));
    RIS_CUDA(cudaEventCreateWithFlags(&evP, cudaEventDisableTiming));
    RIS_CUDA(cudaEventCreateWithFlags(&evC, cudaEventDisableTiming));
    RIS_CUDA(cudaEventCreateWithFlags(&evM, cudaEventDisableTiming));
  }
  if (pin_n < 2 * (size_t)std::max(pl.npair, 1)) {
    if (pin) RIS_CUDA(cudaFreeHost(pin));
    pin = nullptr;
    pin_n = 2 * (size_t)std::max(pl.npair, 1);
    RIS_ALLOC(cudaMallocHost((void**)&pin, sizeof(int) * pin_n));
  }
  // the metric factors (two-centre integrals, Cholesky, inverse) depend on
  // the auxiliary shells only: they run on st3 beside the three-centre
  // integrals (buffers allocated on st first)
  MU.ensure((size_t)nU * nU, st);
  dMU.ensure(3 * (size_t)nU * nU, st);
  if (!d_info) RIS_ALLOC(cudaMallocAsync((void**)&d_info, sizeof(int) * 2, st));
  LJinv.ensure((size_t)nJ * nJ, st);
  LKinv.ensure((size_t)nK * nK, st);
  w1.ensure((size_t)std::max(nJ, nK) * std::max(nJ, nK), st);
  RIS_CUDA(cudaEventRecord(evP, st));
  RIS_CUDA(cudaStreamWaitEvent(st3, evP, 0));
  if (pl.npair > 0) {
    RIS_CUDA(cudaMemcpyAsync(pin, pl.a, sizeof(int) * pl.npair, cudaMemcpyDeviceToHost, st3));
    RIS_CUDA(cudaMemcpyAsync(pin + pl.npair, pl.b, sizeof(int) * pl.npair, cudaMemcpyDeviceToHost, st3));
  }
  RIS_CUDA(cudaEventRecord(evC, st3));
  int2c(aux, xyz.p, MU.p, dMU.p, st3);
  for (int set = 0; set < 2; set++) {
    const int n = set == 0 ? nJ : nK;
    const int* map = set == 0 ? d_jU : d_kU;
    k_gather_sq<<<cdiv(n * n, 256), 256, 0, st3>>>(MU.p, nU, map, n, w1.p);
    RIS_CHECK_LAUNCH();
    cholesky(w1.p, n, d_info + set, st3);
    tri_inverse(w1.p, set == 0 ? LJinv.p : LKinv.p, n, st3);
  }
  RIS_CUDA(cudaEventRecord(evM, st3));
  // integrals: dense [mu][nu][P], or (streamed form) on the screened pairs
  // only, after the metric factors are known
  const int nao_ = ao.nfun;
  streamed = want_streamed(nao_);
  if (!streamed) {
    TJ.ensure((size_t)nao_ * nao_ * nJ, st);
    TK.ensure((size_t)nao_ * nao_ * nK, st);
    RIS_CUDA(cudaMemsetAsync(TJ.p, 0, sizeof(double) * (size_t)nao_ * nao_ * nJ, st));
    RIS_CUDA(cudaMemsetAsync(TK.p, 0, sizeof(double) * (size_t)nao_ * nao_ * nK, st));
    int3c(ao, aux, pl, xyz.p, nJ, nK, TJ.p, TK.p, st);
  } else {
    TJ.release();
    TK.release();
    D.release();
    Df.release();
  }
  RIS_CUDA(cudaStreamWaitEvent(st, evM, 0));
  RIS_CUDA(cudaEventSynchronize(evC));
  h_pa.assign(pin, pin + pl.npair);
  h_pb.assign(pin + pl.npair, pin + 2 * (size_t)pl.npair);
  partners_from_host_pairs();
  int info[2];
  RIS_CUDA(cudaMemcpyAsync(info, d_info, sizeof(info), cudaMemcpyDeviceToHost, st));
  RIS_CUDA(cudaStreamSynchronize(st));
  RIS_REQUIRE(info[0] == 0 && info[1] == 0, RIS_ERR_METRIC_NOT_PD,
              "auxiliary metric is not positive definite (pivot " +
                  std::to_string(info[0] ? info[0] : info[1]) + ")");
  nao = nao_;
  if (streamed) setup_streamed();
  stage = 1;
  if (opt.deriv_prefetch && st2 && !streamed) {  // derivative integrals behind the B build and Davidson
    RIS_CUDA(cudaEventRecord(evA, st));
    RIS_CUDA(cudaStreamWaitEvent(st2, evA, 0));
    start_D(st2);
    RIS_CUDA(cudaEventRecord(evD, st2));
    D_pending = true;
    have_D = true;
  }
}

void Engine::build_B(int nao_, int nmo_, int nocc_, const double* Cin, const double* eps_in) {
  RIS_REQUIRE(stage >= 1, RIS_ERR_STATE, "ris_build_B before ris_build_aux");
  RIS_REQUIRE(nao_ == ao.nfun, RIS_ERR_ARG, "nao does not match the AO basis");
  RIS_REQUIRE(nmo_ <= nao_, RIS_ERR_ARG, "nmo must not exceed nao");
  RIS_REQUIRE(nocc_ > 0 && nocc_ < nmo_, RIS_ERR_ARG, "need 0 < nocc < nmo");
  RIS_REQUIRE(Cin && eps_in, RIS_ERR_ARG, "null pointer");
  stage = 1;
  // active MO range: all MOs, or the energy window around the frontier
  // orbitals (a contiguous column range [i0, a1) of C)
  int i0 = 0, a1 = nmo_;
  if (opt.mo_window > 0.0) {
    std::vector<double> he(nmo_);
    copy_to_host(he.data(), eps_in, nmo_, st);
    for (int i = 1; i < nmo_; i++)
      RIS_REQUIRE(i == nocc_ || he[i] >= he[i - 1], RIS_ERR_ARG,
                  "mo_window needs orbital energies sorted within the occupied and virtual blocks");
    const double lo = he[nocc_ - 1] - opt.mo_window, hi = he[nocc_] + opt.mo_window;
    while (i0 < nocc_ - 1 && he[i0] < lo) i0++;
    while (a1 > nocc_ + 1 && he[a1 - 1] > hi) a1--;
  }
  first_occ = i0;
  nmo = a1 - i0;
  nocc = nocc_ - i0;
  nvir = nmo - nocc;
  const int o = nocc, v = nvir, n = nao;
  const long long nov = (long long)o * v;
  C.ensure((size_t)n * nmo, st);
  eps.ensure(nmo, st);
  de.ensure(nov, st);
  if (i0 == 0 && a1 == nmo_) {
    copy_in(C.p, Cin, (size_t)n * nmo, st);
    copy_in(eps.p, eps_in, nmo, st);
  } else {  // columns i0 .. a1-1 of C [nao][nmo_]
    RIS_CUDA(cudaMemcpy2DAsync(C.p, sizeof(double) * nmo, Cin + i0, sizeof(double) * nmo_,
                               sizeof(double) * nmo, n, cudaMemcpyDefault, st));
    copy_in(eps.p, eps_in + i0, nmo, st);
  }
  k_orb_diff<<<cdiv(nov, 256), 256, 0, st>>>(eps.p, o, v, de.p);
  RIS_CHECK_LAUNCH();
  if (streamed) {
    build_B_streamed();
    stage = 2;
    return;
  }
  const double* Co = C.p;
  const double* Cv = C.p + o;
  // Coulomb: H[i][nu][P] = sum_mu C_mu,i T[mu][nu][P]; B[i][a][P]; B L^-T
  // (mixed form: H as [nu][i][P], both transforms FP64-accurate on the
  // tensor cores)
  const bool emu = opt.precision == RIS_MIXED && opt.emu_f64;
  w2.ensure((size_t)o * n * std::max(nJ, nK), st);
  w3.ensure((size_t)std::max(nov, (long long)o * o) * std::max(nJ, nK), st);
  if (emu) {
    coulomb_emu(w2.p, w3.p);
  } else {
    dgemm(true, false, o, n * nJ, n, 1.0, Co, nmo, TJ.p, n * nJ, 0.0, w2.p, n * nJ, st);
    GemmBatch bt;
    bt.nb1 = o;
    bt.sB1 = (long long)n * nJ;
    bt.sC1 = (long long)v * nJ;
    dgemm(true, false, v, nJ, n, 1.0, Cv, nmo, w2.p, nJ, 0.0, w3.p, nJ, st, bt);
  }
  BJ.ensure((size_t)nov * nJ, st);
  if (emu) {  // B[(i,a)][R] = sum_P W[(i,a)][P] L_J^-1[R][P]
    EmuEpilogue e;
    e.c64 = BJ.p; e.rs = nJ; e.cs = 1;
    emu_abt((int)nov, nJ, nJ, w3.p, nJ, 1, LJinv.p, nJ, 1, e);
  } else {
    dgemm(false, true, (int)nov, nJ, nJ, 1.0, w3.p, nJ, LJinv.p, nJ, 0.0, BJ.p, nJ, st);
  }
  // exchange: oo and ov from C_o^T T^K, vv from C_v^T T^K
  const double* HK = w2.p;
  if (d_kJ) {  // C_o^T T^K: columns of C_o^T T^J
    w5.ensure((size_t)o * n * nK, st);
    const long long rows = (long long)o * n;
    k_gather_cols<<<(unsigned)cdiv(rows * nK, 256), 256, 0, st>>>(w2.p, rows, nJ, d_kJ, nK, w5.p,
                                                                  emu ? n : 0, o);
    RIS_CHECK_LAUNCH();
    HK = w5.p;
  } else {
    dgemm(true, false, o, n * nK, n, 1.0, Co, nmo, TK.p, n * nK, 0.0, w2.p, n * nK, st);
  }
  {
    GemmBatch bt;
    bt.nb1 = o;
    bt.sB1 = (long long)n * nK;
    bt.sC1 = (long long)o * nK;
    dgemm(true, false, o, nK, n, 1.0, Co, nmo, HK, nK, 0.0, w3.p, nK, st, bt);
  }
  BKoo.ensure((size_t)o * o * nK, st);
  dgemm(false, true, o * o, nK, nK, 1.0, w3.p, nK, LKinv.p, nK, 0.0, BKoo.p, nK, st);
  cKoo.ensure((size_t)o * o * nK, st);
  dgemm(false, false, o * o, nK, nK, 1.0, BKoo.p, nK, LKinv.p, nK, 0.0, cKoo.p, nK, st);
  if (opt.rpa) {
    GemmBatch bt;
    bt.nb1 = o;
    bt.sB1 = (long long)n * nK;
    bt.sC1 = (long long)v * nK;
    dgemm(true, false, v, nK, n, 1.0, Cv, nmo, HK, nK, 0.0, w3.p, nK, st, bt);
    w4.ensure((size_t)nov * nK, st);
    dgemm(false, true, (int)nov, nK, nK, 1.0, w3.p, nK, LKinv.p, nK, 0.0, w4.p, nK, st);  // [i][a][R]
    cKov.ensure((size_t)nov * nK, st);
    dgemm(false, false, (int)nov, nK, nK, 1.0, w4.p, nK, LKinv.p, nK, 0.0, cKov.p, nK, st);
    BKovR.ensure((size_t)nov * nK, st);
    transpose_last2(w4.p, 1, (int)nov, nK, BKovR.p, st);  // [R][ia]
    cKovP.ensure((size_t)nov * nK, st);
    transpose_last2(cKov.p, 1, (int)nov, nK, cKovP.p, st);  // [P][ia]
  }
  w4.ensure((size_t)v * v * nK, st);
  if (opt.precision == RIS_MIXED && !opt.refine) {
    build_Kvv_tc(w4.p);  // B[a][b][R]
  } else {
    w2.ensure((size_t)v * n * nK, st);
    dgemm(true, false, v, n * nK, n, 1.0, Cv, nmo, TK.p, n * nK, 0.0, w2.p, n * nK, st);
    w3.ensure((size_t)v * v * nK, st);
    GemmBatch bt;
    bt.nb1 = v;
    bt.sB1 = (long long)n * nK;
    bt.sC1 = (long long)v * nK;
    dgemm(true, false, v, nK, n, 1.0, Cv, nmo, w2.p, nK, 0.0, w3.p, nK, st, bt);
    dgemm(false, true, v * v, nK, nK, 1.0, w3.p, nK, LKinv.p, nK, 0.0, w4.p, nK, st);  // B[a][b][R]
  }
  cKvv.ensure((size_t)v * v * nK, st);
  if (emu) {  // c[(a,b)][Q] = sum_R B[(a,b)][R] L_K^-1[R][Q]
    EmuEpilogue e;
    e.c64 = cKvv.p; e.rs = nK; e.cs = 1;
    emu_abt(v * v, nK, nK, w4.p, nK, 1, LKinv.p, 1, nK, e);
  } else {
    dgemm(false, false, v * v, nK, nK, 1.0, w4.p, nK, LKinv.p, nK, 0.0, cKvv.p, nK, st);
  }
  BKvvD.ensure((size_t)v * v * nK, st);
  transpose_last2(w4.p, v, v, nK, BKvvD.p, st);  // [b][R][a]
  if (opt.precision == RIS_MIXED) prepare_mixed();
  stage = 2;
}

// FP32 hi/lo operands of the exchange products (Eq. A_matrix, (ij|ab) term)
void Engine::prepare_mixed() {
  const int o = nocc, v = nvir, n = nao;
  const int lo4 = ld4(o), lv4 = ld4(v);
  if (!d_tcerr) {
    RIS_ALLOC(cudaMallocAsync((void**)&d_tcerr, sizeof(int), st));
    RIS_CUDA(cudaMemsetAsync(d_tcerr, 0, sizeof(int), st));
  }
  BooH.ensure((size_t)o * nK * lo4, st);
  BooL.ensure((size_t)o * nK * lo4, st);
  // per i: [j][R] -> [R][j]
  split_f64_t(BKoo.p, o, nK, nK, BooH.p, BooL.p, lo4, st, o, (long long)o * nK, (long long)nK * lo4);
  BvvH.ensure((size_t)v * nK * lv4, st);
  BvvL.ensure((size_t)v * nK * lv4, st);
  // BKvvD [b][R][a] = [a][R][b] by symmetry; rows (a,R), b padded
  split_f64(BKvvD.p, v * nK, v, v, BvvH.p, BvvL.p, lv4, st);
  // fitting coefficients for Gamma: c^vv[a][b][P] -> [P][b][a] (symmetric in a,b)
  w3.ensure((size_t)v * v * nK, st);
  transpose_last2(cKvv.p, 1, v * v, nK, w3.p, st);  // [P][(a,b)]
  cvvH.ensure((size_t)nK * v * lv4, st);
  cvvL.ensure((size_t)nK * v * lv4, st);
  split_f64(w3.p, nK * v, v, v, cvvH.p, cvvL.p, lv4, st);
  cKooP.ensure((size_t)o * o * nK, st);
  transpose_last2(cKoo.p, 1, o * o, nK, cKooP.p, st);  // [P][i][k]
  cooH.ensure((size_t)nK * o * lo4, st);
  cooL.ensure((size_t)nK * o * lo4, st);
  split_f64(cKooP.p, nK * o, o, o, cooH.p, cooL.p, lo4, st);
  // C_o and C_v as [mu][p]
  CoH.ensure((size_t)n * lo4, st);
  CoL.ensure((size_t)n * lo4, st);
  split_f64(C.p, n, o, nmo, CoH.p, CoL.p, lo4, st);
  CvH.ensure((size_t)n * lv4, st);
  CvL.ensure((size_t)n * lv4, st);
  split_f64(C.p + o, n, v, nmo, CvH.p, CvL.p, lv4, st);
}

// One tensor-core GEMM with split operands; helper for the mixed path.
static void tcg(int M, int N, int K, const float* ah, const float* al, int lda, const float* bh,
                const float* bl, int ldb, long long bsb, int nb, const TcEpilogue& e, int* err,
                cudaStream_t st, long long bsa = 0, int nba = 1) {
  TcOperand A, B;
  A.hi = ah; A.lo = al; A.rows = M; A.ld = lda; A.bstride = bsa; A.nb = nba;
  B.hi = bh; B.lo = bl; B.rows = N; B.ld = ldb; B.bstride = bsb;
  B.nb = (nb > 1 && bsb != 0) ? nb : 1;  // bsb == 0: one B shared by every batch
  tc_gemm(M, N, K, A, B, nb, e, err, st);
}
static TcEpilogue ep_split(float* h, float* l, long long rs, long long cs = 1, long long bsc = 0) {
  TcEpilogue e;
  e.mode = kOutSplit; e.chi = h; e.clo = l; e.rs = rs; e.cs = cs; e.bsc = bsc;
  return e;
}
static TcEpilogue ep_f64(double* c, long long rs, long long bsc = 0, double alpha = 1.0,
                         double beta = 0.0, long long cs = 1) {
  TcEpilogue e;
  e.mode = kOutF64; e.c64 = c; e.rs = rs; e.cs = cs; e.bsc = bsc; e.alpha = alpha; e.beta = beta;
  return e;
}

// Mixed precision, Coulomb transforms (ia|P)_J = sum_mu,nu C_mu,i C_nu,a
// (mu nu|P) as FP64-accurate products on the FP16 tensor cores (exact
// operand splitting, gemm_emu.cu).  The J metric is ill-conditioned and the
// MO transforms cancel heavily, so these stay at FP64 accuracy.
// Transform 1: H[(nu,P)][i] = sum_mu T[(nu,P)][mu] C_o[mu][i], stored as
// H[nu][i][P] (T symmetric in mu, nu; read through (mu nu|P) = T[mu][nu][P]);
// transform 2: W[(i,P)][a] = sum_nu H[(i,P)][nu] C_v[nu][a], stored as
// W[i][a][P].
void Engine::coulomb_emu(double* H, double* W) {
  const int o = nocc, v = nvir, n = nao;
  const long long rT = (long long)n * nJ, rH = (long long)o * nJ;
  RIS_REQUIRE(rT < (1ll << 31), RIS_ERR_ARG, "Coulomb transform too large for one product");
  // H[(nu,P)][i]: A[(nu,P)][mu] = T[mu][(nu,P)], B[i][mu] = C[mu][i]
  EmuEpilogue e1;
  e1.c64 = H; e1.rin = nJ; e1.rld = rH; e1.rs = 1; e1.cs = nJ;
  emu_abt((int)rT, o, n, TJ.p, 1, rT, C.p, 1, nmo, e1);
  // W[(i,P)][a]: A[(i,P)][nu] = H[nu][(i,P)], B[a][nu] = C[nu][o + a]
  EmuEpilogue e2;
  e2.c64 = W; e2.rin = nJ; e2.rld = (long long)v * nJ; e2.rs = 1; e2.cs = nJ;
  emu_abt((int)rH, v, n, H, 1, rH, C.p + o, 1, nmo, e2);
}

void Engine::emu_abt(int M, int N, int K, const double* A, long long rsA, long long ksA,
                     const double* B, long long rsB, long long ksB, const EmuEpilogue& ep) {
  if (!d_tcerr) {
    RIS_ALLOC(cudaMallocAsync((void**)&d_tcerr, sizeof(int), st));
    RIS_CUDA(cudaMemsetAsync(d_tcerr, 0, sizeof(int), st));
  }
  const int lk = ld8(K);
  SBuf<__half> sA((size_t)kEmuSlices * M * lk, st), sB((size_t)kEmuSlices * N * lk, st);
  SBuf<int> eA(M, st), eB(N, st);
  EmuOperand a, b;
  a.s = sA.p; a.e = eA.p;
  b.s = sB.p; b.e = eB.p;
  emu_slice(A, M, K, rsA, ksA, a, st);
  emu_slice(B, N, K, rsB, ksB, b, st);
  emu_gemm(M, N, a, b, ep, d_tcerr, st);
}

// Mixed precision: (ab|P)_K = sum_mu,nu C_mu,a C_nu,b (mu nu|P) by two
// 3xTF32 tensor-core transforms, then B = (ab|P) L_K^-T by a third (out
// [a][b][R]; the K metric is well conditioned, its smallest eigenvalue about
// 0.05).  Half transform 1: H[a][P][nu] = sum_mu C_v^T[a][mu] T[(P,nu)][mu]
// with T[(P,nu)][mu] = (nu mu|P) (symmetric in mu, nu); transform 2:
// G[a][b][P] = sum_nu C_v^T[b][nu] H[(a,P)][nu].
void Engine::build_Kvv_tc(double* out) {
  const int o = nocc, v = nvir, n = nao;
  const int ldn = ld4(n);
  if (!d_tcerr) {
    RIS_ALLOC(cudaMallocAsync((void**)&d_tcerr, sizeof(int), st));
    RIS_CUDA(cudaMemsetAsync(d_tcerr, 0, sizeof(int), st));
  }
  SBuf<float> Th((size_t)nK * n * ldn, st), Tl((size_t)nK * n * ldn, st);
  SBuf<float> CvTh((size_t)v * ldn, st), CvTl((size_t)v * ldn, st);
  SBuf<float> Hh((size_t)v * nK * ldn, st), Hl((size_t)v * nK * ldn, st);
  split_f64_tpad(TK.p, (long long)n * n, nK, n, ldn, Th.p, Tl.p, st);  // [P][nu][mu]
  split_f64_t(C.p + o, n, v, nmo, CvTh.p, CvTl.p, ldn, st);            // [a][mu]
  {
    TcEpilogue e = ep_split(Hh.p, Hl.p, (long long)nK * ldn);
    e.cin = n;
    e.cld = ldn;
    tcg(v, nK * n, n, CvTh.p, CvTl.p, ldn, Th.p, Tl.p, ldn, 0, 1, e, d_tcerr, st);
  }
  // G[b][(a,P)] = sum_nu C_v^T[b][nu] H[(a,P)][nu], stored split as
  // [a][b][P] (P padded to lk, zero) so that it is the K-major operand of the
  // metric product; consecutive lanes of the epilogue write consecutive P
  const int lk = ld4(nK);
  SBuf<float> Gh((size_t)v * v * lk, st, true), Gl((size_t)v * v * lk, st, true);
  {
    TcEpilogue e = ep_split(Gh.p, Gl.p, lk);
    e.cin = nK;
    e.cld = (long long)v * lk;
    tcg(v, v * nK, n, CvTh.p, CvTl.p, ldn, Hh.p, Hl.p, ldn, 0, 1, e, d_tcerr, st);
  }
  // out[(a,b)][R] = sum_P G[a][b][P] L^-1[R][P] (3xTF32, one GEMM over every (a, b))
  SBuf<float> Lh((size_t)nK * lk, st), Ll((size_t)nK * lk, st);
  split_f64(LKinv.p, nK, nK, nK, Lh.p, Ll.p, lk, st);
  tcg(v * v, nK, nK, Gh.p, Gl.p, lk, Lh.p, Ll.p, lk, 0, 1, ep_f64(out, nK), d_tcerr, st);
  // restore the exact a <-> b symmetry that rounding broke (A must stay symmetric)
  k_sym_pairs<<<cdiv((long long)v * v * nK, 256), 256, 0, st>>>(out, v, nK);
  RIS_CHECK_LAUNCH();
  (void)o;
}

void Engine::gamma_K_mixed(const float* USh, const float* USl, const float* VSh, const float* VSl,
                           const float* WUh, const float* WUl, const float* WVh, const float* WVl,
                           double f, double* Gam, float* Gam32, double* Om) {
  const int o = nocc, v = nvir, nn = nao;
  const int lv4 = ld4(v), lo4 = ld4(o), kp = ld4(2 * o);
  // Z[P][j][b] = sum_a U[j][a] c^vv[P][b][a]   (one GEMM, columns (P, b))
  SBuf<float> ZH((size_t)nK * o * lv4, st, true), ZL((size_t)nK * o * lv4, st, true);
  {
    TcEpilogue e = ep_split(ZH.p, ZL.p, lv4);
    e.cin = v;
    e.cld = (long long)o * lv4;
    tcg(o, nK * v, v, USh, USl, lv4, cvvH.p, cvvL.p, lv4, 0, 1, e, d_tcerr, st);
  }
  // G[P][k][j] = sum_b V[k][b] Z[P][j][b]   (batch P, coalesced rows)
  SBuf<float> GH((size_t)nK * o * lo4, st, true), GL((size_t)nK * o * lo4, st, true);
  tcg(o, o, v, VSh, VSl, lv4, ZH.p, ZL.p, lv4, (long long)o * lv4, nK,
      ep_split(GH.p, GL.p, lo4, 1, (long long)o * lo4), d_tcerr, st);
  // M1[mu][P][k'] : k' < o  sum_i Q_U[i][mu] c^oo[P][i][k]
  //                 k' >= o sum_j C_o[mu][j] G[P][k][j]
  // each one GEMM over the columns (P, k)
  SBuf<float> MH((size_t)nn * nK * kp, st, true), ML((size_t)nn * nK * kp, st, true);
  {
    TcEpilogue e = ep_split(MH.p, ML.p, (long long)nK * kp);
    e.cin = o;
    e.cld = kp;
    tcg(nn, nK * o, o, WUh, WUl, kp, cooH.p, cooL.p, lo4, 0, 1, e, d_tcerr, st);
    e.chi = MH.p + o;
    e.clo = ML.p + o;
    tcg(nn, nK * o, o, CoH.p, CoL.p, lo4, GH.p, GL.p, lo4, 0, 1, e, d_tcerr, st);
  }
  // Gamma[mu][nu][P] += f sum_k' W_V[nu][k'] M1[mu][P][k']: one GEMM, rows nu,
  // columns (mu, P)
  {
    TcEpilogue e = Gam32 ? TcEpilogue() : ep_f64(Gam, nK, 0, f, 1.0);
    if (Gam32) {  // sole writer of the FP32 G^K: plain stores, no read-modify-write
      e.mode = kOutF32;
      e.c32 = Gam32;
      e.alpha = f;
      e.beta = 0.0;
    }
    e.rs = nK;
    e.cin = nK;
    e.cld = (long long)nn * nK;
    tcg(nn, nn * nK, 2 * o, WVh, WVl, kp, MH.p, ML.p, kp, 0, 1, e, d_tcerr, st);
  }
  // Omega[A][B] += f sum_{k,j} c^oo[A][k][j] G[B][k][j]
  tcg(nK, nK, o * lo4, cooH.p, cooL.p, o * lo4, GH.p, GL.p, o * lo4, 0, 1, ep_f64(Om, nU, 0, f, 1.0),
      d_tcerr, st);
}

// out = alpha * K1 + beta * out with K1 the (ij|ab) exchange contraction of
// the nvec vectors Z, as two 3xTF32 GEMMs:
//   Y[vec][(i,R)][b] = sum_j B^K_oo[(i,R)][j] Z[vec][j][b]
//   K1[(vec,i)][a]   = sum_{(R,b)} Y[(vec,i)][(R,b)] B^K_vv[a][(R,b)]
void Engine::apply_exchange_mixed(const double* Z, int nvec, double* out, double alpha,
                                  double beta) {
  const int o = nocc, v = nvir;
  const long long nov = (long long)o * v;
  const int lo4 = ld4(o), lv4 = ld4(v);
  XtH.ensure((size_t)nvec * v * lo4, st);
  XtL.ensure((size_t)nvec * v * lo4, st);
  split_f64_t(Z, o, v, v, XtH.p, XtL.p, lo4, st, nvec, nov, (long long)v * lo4);
  // occupied orbitals per pass: all of them while Y stays below 3 Gi floats
  // (per half), else blocks of ib (each pass reads B^K_vv once more)
  const size_t per_i = (size_t)nvec * nK * lv4;
  int ib = o;
  if (opt.occ_block > 0)
    ib = std::min(o, opt.occ_block);
  else if (per_i * o > ((size_t)3 << 30))
    ib = std::max(1, (int)(((size_t)3 << 30) / per_i));
  const size_t ysz = per_i * ib;
  if (YH.n < ysz) {
    YH.ensure(ysz, st);
    YL.ensure(ysz, st);
  }
  for (int i0 = 0; i0 < o; i0 += ib) {
    const int ni = std::min(ib, o - i0);
    TcOperand A, B;
    A.hi = BooH.p + (size_t)i0 * nK * lo4;
    A.lo = BooL.p + (size_t)i0 * nK * lo4;
    A.rows = ni * nK;
    A.ld = lo4;
    B.hi = XtH.p;
    B.lo = XtL.p;
    B.rows = v;
    B.ld = lo4;
    B.bstride = (long long)v * lo4;
    B.nb = nvec;
    TcEpilogue e1;
    e1.mode = kOutSplit;
    e1.chi = YH.p;
    e1.clo = YL.p;
    e1.rs = lv4;
    e1.bsc = (long long)ni * nK * lv4;
    tc_gemm(ni * nK, v, o, A, B, nvec, e1, d_tcerr, st);
    TcOperand A2, B2;
    A2.hi = YH.p;
    A2.lo = YL.p;
    A2.rows = nvec * ni;
    A2.ld = nK * lv4;
    B2.hi = BvvH.p;
    B2.lo = BvvL.p;
    B2.rows = v;
    B2.ld = nK * lv4;
    TcEpilogue e2;
    e2.mode = kOutF64;
    e2.c64 = out + (size_t)i0 * v;  // row (vec, i) -> out[vec][i0 + i]
    e2.rs = v;
    if (ni < o) {
      e2.rin = ni;
      e2.rld = nov;
    }
    e2.alpha = alpha;
    e2.beta = beta;
    tc_gemm(nvec * ni, v, nK * lv4, A2, B2, 1, e2, d_tcerr, st);
  }
}

void Engine::apply_A_mixed(const double* Xin, int nvec, double* out) {
  const long long nov = (long long)nocc * nvir;
  // Coulomb, FP64-accurate: out = 2 (X B^J) B^J^T (double-FP32 with subspace_ff)
  w5.ensure((size_t)nvec * std::max(nJ, 1), st);
  const bool ff = opt.subspace_ff != 0;
  gemm_sub(ff, false, false, nvec, nJ, (int)nov, 1.0, Xin, (int)nov, BJ.p, nJ, 0.0, w5.p, nJ, st);
  gemm_sub(ff, false, true, nvec, (int)nov, nJ, 2.0, w5.p, nJ, BJ.p, nJ, 0.0, out, (int)nov, st);
  apply_exchange_mixed(Xin, nvec, out, -opt.cx, 1.0);
  k_add_diag<<<cdiv(nov * nvec, 256), 256, 0, st>>>(de.p, Xin, nov, nvec, out);
  RIS_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ A products
// out[n] = A X[n] for TDA (Eq. A_matrix with the ris kernel)
void Engine::apply_A_tda(const double* Xin, int nvec, double* out) {
  const int o = nocc, v = nvir;
  const long long nov = (long long)o * v;
  w5.ensure((size_t)nvec * std::max(nJ, 1), st);
  dgemm(false, false, nvec, nJ, (int)nov, 1.0, Xin, (int)nov, BJ.p, nJ, 0.0, w5.p, nJ, st);
  dgemm(false, true, nvec, (int)nov, nJ, 2.0, w5.p, nJ, BJ.p, nJ, 0.0, out, (int)nov, st);
  w6.ensure((size_t)nvec * o * nK * v, st);
  {
    GemmBatch bt;
    bt.nb1 = nvec;
    bt.sA1 = nov;
    bt.sC1 = (long long)o * nK * v;
    dgemm(false, false, o, nK * v, v, 1.0, Xin, v, BKvvD.p, nK * v, 0.0, w6.p, nK * v, st, bt);
  }
  {
    GemmBatch bt;
    bt.nb1 = nvec;
    bt.sB1 = (long long)o * nK * v;
    bt.sC1 = nov;
    dgemm(false, false, o, v, o * nK, -opt.cx, BKoo.p, o * nK, w6.p, v, 1.0, out, v, st, bt);
  }
  k_add_diag<<<cdiv(nov * nvec, 256), 256, 0, st>>>(de.p, Xin, nov, nvec, out);
  RIS_CHECK_LAUNCH();
}

void Engine::apply(int nvec, const double* Xh, double* out, double* out2) {
  RIS_REQUIRE(stage >= 2, RIS_ERR_STATE, "ris_apply before ris_build_B");
  RIS_REQUIRE(nvec >= 1 && Xh && out, RIS_ERR_ARG, "bad ris_apply arguments");
  RIS_REQUIRE((out2 != nullptr) == (opt.rpa != 0), RIS_ERR_ARG, "out2 must be given exactly for RPA");
  const size_t n = (size_t)nvec * nocc * nvir;
  SBuf<double> x(n, st), y(n, st), z;
  copy_in(x.p, Xh, n, st);
  if (opt.rpa) {
    z.ensure(n, st);
    apply_ApB_AmB(x.p, nvec, y.p, z.p);
    copy_out(out2, z.p, n, st);
  } else if (opt.precision == RIS_MIXED) {
    apply_A_mixed(x.p, nvec, y.p);
  } else {
    apply_A_tda(x.p, nvec, y.p);
  }
  copy_out(out, y.p, n, st);
  RIS_CUDA(cudaStreamSynchronize(st));
}

// (ij|ab) and (ib|ja) exchange contractions (Eqs. A_matrix, B_matrix):
//   K1[n][i][a] = sum_{R,j,b} B^K_ij,R Z_n[j][b] B^K_ab,R
//   K2[n][i][a] = sum_{R,j,b} B^K_ib,R Z_n[j][b] B^K_ja,R
void Engine::exchange_terms(const double* Z, int nvec, double* K1, double* K2, bool mixed) {
  const int o = nocc, v = nvir;
  const long long nov = (long long)o * v;
  if (mixed) {
    apply_exchange_mixed(Z, nvec, K1, 1.0, 0.0);
  } else {
    w6.ensure((size_t)nvec * o * nK * v, st);
    GemmBatch bt;
    bt.nb1 = nvec;
    bt.sA1 = nov;
    bt.sC1 = (long long)o * nK * v;
    dgemm(false, false, o, nK * v, v, 1.0, Z, v, BKvvD.p, nK * v, 0.0, w6.p, nK * v, st, bt);
    GemmBatch b2;
    b2.nb1 = nvec;
    b2.sB1 = (long long)o * nK * v;
    b2.sC1 = nov;
    dgemm(false, false, o, v, o * nK, 1.0, BKoo.p, o * nK, w6.p, v, 0.0, K1, v, st, b2);
  }
  // Y1[n][i][R][j] = sum_b B^K_ib,R Z_n[j][b];  K2_n = Y1_n . B^K as [(R,j)][a]
  SBuf<double> Y1((size_t)nvec * o * nK * o, st);
  GemmBatch bt;
  bt.nb1 = nvec;
  bt.nb2 = nK;
  bt.sA1 = 0;
  bt.sA2 = nov;
  bt.sB1 = nov;
  bt.sB2 = 0;
  bt.sC1 = (long long)o * nK * o;
  bt.sC2 = o;
  dgemm(false, true, o, o, v, 1.0, BKovR.p, v, Z, v, 0.0, Y1.p, nK * o, st, bt);
  GemmBatch b2;
  b2.nb1 = nvec;
  b2.sA1 = (long long)o * nK * o;
  b2.sC1 = nov;
  dgemm(false, false, o, v, nK * o, 1.0, Y1.p, nK * o, BKovR.p, v, 0.0, K2, v, st, b2);
}

void Engine::apply_ApB_AmB(const double* Z, int nvec, double* outP, double* outM) {
  const long long nov = (long long)nocc * nvir;
  const bool mixed = opt.precision == RIS_MIXED;
  w5.ensure((size_t)nvec * std::max(nJ, 1), st);
  dgemm(false, false, nvec, nJ, (int)nov, 1.0, Z, (int)nov, BJ.p, nJ, 0.0, w5.p, nJ, st);
  dgemm(false, true, nvec, (int)nov, nJ, 1.0, w5.p, nJ, BJ.p, nJ, 0.0, outP, (int)nov, st);
  SBuf<double> K1((size_t)nvec * nov, st), K2((size_t)nvec * nov, st);
  exchange_terms(Z, nvec, K1.p, K2.p, mixed);
  k_rpa_combine<<<cdiv(nov * nvec, 256), 256, 0, st>>>(de.p, Z, K1.p, K2.p, nov, nvec, opt.cx, outP, outM);
  RIS_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ Davidson (TDA)
void Engine::davidson_tda(int ns, const double* guess) {
  if (opt.precision != RIS_MIXED) {
    dav_core(ns, guess, guess ? ns : 0, false, opt.conv_tol, true);
    return;
  }
  bool ok = true;
  const double tolm = std::max(opt.conv_tol, opt.mixed_tol);
  struct ReleaseY {  // streamed form: the exchange work space is large; give it back
    Engine& e;
    ~ReleaseY() {
      if (e.streamed) {
        e.YH.release();
        e.YL.release();
      }
    }
  } release_y{*this};
  dav_core(ns, guess, guess ? ns : 0, true, tolm, true, streamed ? nullptr : &ok);
  if (!ok) {
    // the 3xTF32 products stalled above the tolerance: continue from the
    // current vectors with FP64 products to the same tolerance
    SBuf<double> g((size_t)ns * nocc * nvir, st);
    RIS_CUDA(cudaMemcpyAsync(g.p, X.p, sizeof(double) * g.n, cudaMemcpyDeviceToDevice, st));
    const double s4 = stats[4], s5 = stats[5];
    dav_core(ns, g.p, ns, false, tolm);
    stats[6] = stats[4];
    stats[4] += s4;
    stats[5] += s5;
  }
  if (opt.refine) {
    SBuf<double> g((size_t)ns * nocc * nvir, st);
    RIS_CUDA(cudaMemcpyAsync(g.p, X.p, sizeof(double) * g.n, cudaMemcpyDeviceToDevice, st));
    const double s4 = stats[4], s5 = stats[5];
    dav_core(ns, g.p, ns, false, opt.conv_tol);
    stats[6] = stats[4];  // FP64 products of the refinement
    stats[4] += s4;
    stats[5] += s5;
  }
  int h_err = 0;
  RIS_CUDA(cudaMemcpyAsync(&h_err, d_tcerr, sizeof(int), cudaMemcpyDeviceToHost, st));
  RIS_CUDA(cudaStreamSynchronize(st));
  RIS_REQUIRE(h_err == 0, RIS_ERR_TIMEOUT, "a tensor-core GEMM pipeline wait timed out");
}

// M = D - s + f B^J B^J^T (orbital-energy differences plus the Coulomb part
// of A (f = 2, Eq. A_matrix) or of A + B (f = 4, Eq. Z_vector)), inverted
// exactly by the Woodbury identity with D' = D - s:
//   M^-1 r = D'^-1 r - f D'^-1 B (I + f B^T D'^-1 B)^-1 B^T D'^-1 r.
// shifted: s just below the smallest difference (Davidson: one shift for
// all states); otherwise s = 0.  The capacitance matrix (nJ x nJ) is
// Cholesky-factored once; each application is three skinny GEMMs.
void CoulPrecond::setup(Engine& e, bool shifted, double f_, int nmax) {
  const long long n = (long long)e.nocc * e.nvir;
  const int nJ = e.nJ;
  cudaStream_t st = e.st;
  f = f_;
  dinv.ensure(n, st);
  capinv.ensure((size_t)nJ * nJ, st);
  pY.ensure((size_t)nmax * nJ, st);
  pZ.ensure((size_t)nmax * nJ, st);
  pP.ensure((size_t)nmax * n, st);
  // the capacitance matrix B^T D'^-1 B over row blocks of at most 2^27
  // elements of the scaled B (one block for all but the largest systems)
  const long long rblk = std::max(1LL, std::min(n, (1LL << (e.opt.precision == RIS_MIXED ? 26 : 27)) /
                                                       std::max(nJ, 1)));
  SBuf<double> W((size_t)rblk * nJ, st), cap((size_t)nJ * nJ, st), Li((size_t)nJ * nJ, st),
      dm(1, st, true);
  SBuf<int> info(1, st);
  if (shifted) {
    k_min<<<1, 1024, 0, st>>>(e.de.p, n, dm.p);
    RIS_CHECK_LAUNCH();
  }
  // mixed precision: the capacitance matrix only steers the preconditioner
  // (never the converged pairs), so its long-K product runs as a 3xTF32
  // tensor-core GEMM on transposed row blocks
  const bool use_tc = e.opt.precision == RIS_MIXED && e.d_tcerr;
  const int ldr = ld4((int)std::min(rblk, n));
  SBuf<float> capBh, capBl, capWh, capWl;  // transposed splits of one row block
  if (use_tc) {
    capBh.ensure((size_t)nJ * ldr, st);
    capBl.ensure((size_t)nJ * ldr, st);
    capWh.ensure((size_t)nJ * ldr, st);
    capWl.ensure((size_t)nJ * ldr, st);
  }
  for (long long r0 = 0; r0 < n; r0 += rblk) {
    const long long nr = std::min(rblk, n - r0);
    k_precond_setup<<<cdiv(nr * nJ, 256), 256, 0, st>>>(e.de.p, dm.p, r0, nr, shifted ? kPrecondGap : 0.0,
                                                         e.BJ.p, nJ, dinv.p, W.p);
    RIS_CHECK_LAUNCH();
    if (use_tc) {
      const int lr = ld4((int)nr);
      split_f64_t(e.BJ.p + (size_t)r0 * nJ, (int)nr, nJ, nJ, capBh.p, capBl.p, lr, st);  // [P][row]
      split_f64_t(W.p, (int)nr, nJ, nJ, capWh.p, capWl.p, lr, st);
      tcg(nJ, nJ, (int)nr, capBh.p, capBl.p, lr, capWh.p, capWl.p, lr, 0, 1,
          ep_f64(cap.p, nJ, 0, f, r0 == 0 ? 0.0 : 1.0), e.d_tcerr, st);
    } else {
      dgemm(true, false, nJ, nJ, (int)nr, f, e.BJ.p + (size_t)r0 * nJ, nJ, W.p, nJ, r0 == 0 ? 0.0 : 1.0,
            cap.p, nJ, st);
    }
  }
  k_add_identity<<<cdiv(nJ, 128), 128, 0, st>>>(cap.p, nJ);
  RIS_CHECK_LAUNCH();
  cholesky(cap.p, nJ, info.p, st);
  tri_inverse(cap.p, Li.p, nJ, st);
  dgemm(true, false, nJ, nJ, nJ, 1.0, Li.p, nJ, Li.p, nJ, 0.0, capinv.p, nJ, st);
  // mixed precision: 3xTF32 applications when the splits of B^J stay small
  // (a preconditioner only changes the number of iterations)
  tc = use_tc && (double)n * (ld4(nJ) + nJ) * 8.0 < 4.0e9;
  if (tc) {
    const int ln = ld4((int)n), lj = ld4(nJ);
    Bh.ensure((size_t)n * lj, st);
    Bl.ensure((size_t)n * lj, st);
    BTh.ensure((size_t)nJ * ln, st);
    BTl.ensure((size_t)nJ * ln, st);
    Th.ensure((size_t)nmax * ln, st);
    Tl.ensure((size_t)nmax * ln, st);
    Zh.ensure((size_t)nmax * lj, st);
    Zl.ensure((size_t)nmax * lj, st);
    split_f64(e.BJ.p, (int)n, nJ, nJ, Bh.p, Bl.p, lj, st);
    split_f64_t(e.BJ.p, (int)n, nJ, nJ, BTh.p, BTl.p, ln, st);
  }
  int h_info = 0;
  RIS_CUDA(cudaMemcpyAsync(&h_info, info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  RIS_CUDA(cudaStreamSynchronize(st));
  RIS_REQUIRE(h_info == 0, RIS_ERR_ARG, "preconditioner capacitance matrix not positive definite");
}

void CoulPrecond::apply(Engine& e, const double* R, const int* idx, int nt, double* T) {
  const long long n = (long long)e.nocc * e.nvir;
  const int nJ = e.nJ;
  cudaStream_t st = e.st;
  k_precond_scale<<<cdiv(n * nt, 256), 256, 0, st>>>(R, dinv.p, idx, n, nt, T);
  RIS_CHECK_LAUNCH();
  if (tc) {  // the two long products on the 3xTF32 tensor cores
    RIS_REQUIRE(Bh.p && BTh.p && Th.p && Zh.p && nt <= (int)(Zh.n / ld4(nJ)), RIS_ERR_ARG,
                "preconditioner splits missing");
    const int ln = ld4((int)n), lj = ld4(nJ);
    split_f64(T, nt, (int)n, n, Th.p, Tl.p, ln, st);
    tcg(nt, nJ, (int)n, Th.p, Tl.p, ln, BTh.p, BTl.p, ln, 0, 1, ep_f64(pY.p, nJ), e.d_tcerr, st);
    dgemm(false, false, nt, nJ, nJ, 1.0, pY.p, nJ, capinv.p, nJ, 0.0, pZ.p, nJ, st);
    split_f64(pZ.p, nt, nJ, nJ, Zh.p, Zl.p, lj, st);
    tcg(nt, (int)n, nJ, Zh.p, Zl.p, lj, Bh.p, Bl.p, lj, 0, 1, ep_f64(pP.p, n), e.d_tcerr, st);
  } else {
    dgemm(false, false, nt, nJ, (int)n, 1.0, T, (int)n, e.BJ.p, nJ, 0.0, pY.p, nJ, st);
    dgemm(false, false, nt, nJ, nJ, 1.0, pY.p, nJ, capinv.p, nJ, 0.0, pZ.p, nJ, st);
    dgemm(false, true, nt, (int)n, nJ, 1.0, pZ.p, nJ, e.BJ.p, nJ, 0.0, pP.p, (int)n, st);
  }
  k_precond_update<<<cdiv(n * nt, 256), 256, 0, st>>>(T, pP.p, dinv.p, n, nt, f);
  RIS_CHECK_LAUNCH();
}

// Block Davidson for the lowest ns eigenpairs of the TDA A.  Starts from
// unit vectors on the lowest orbital-energy differences, or from nguess
// given vectors (augment: plus unit vectors up to the usual block size);
// products in FP64 or (mixed) with 3xTF32 exchange GEMMs.
void Engine::dav_core(int ns, const double* guess, int nguess, bool mixed, double tol,
                      bool augment, bool* ok) {
  const long long n = (long long)nocc * nvir;
  const int nb0 = (int)std::min<long long>(n, ns + std::min(ns, 8));
  // automatic size: 8 ns, or 4 ns for the mixed phase when the products are
  // cheap (nov <= 2^20): its looser tolerance converges in as many
  // iterations from the smaller subspace, whose FP64 eigensolve (latency-
  // bound, about m^3) then costs far less
  const int mult = mixed && n <= (1LL << 20) ? 4 : 8;
  int maxsp = opt.max_subspace > 0 ? opt.max_subspace : std::max(nb0 + 2 * ns, mult * ns);
  maxsp = (int)std::min<long long>(std::min(maxsp, 256), n);
  RIS_REQUIRE(maxsp >= nb0, RIS_ERR_ARG, "max_subspace smaller than the initial block");
  const int kkeep = std::min(2 * ns, 64);
  SBuf<double> V((size_t)maxsp * n, st), AV((size_t)maxsp * n, st), Hs((size_t)maxsp * maxsp, st),
      S((size_t)64 * maxsp, st), w(64, st), Xr((size_t)ns * n, st), AXr((size_t)ns * n, st),
      Rr((size_t)ns * n, st), T((size_t)ns * n, st), tmp((size_t)std::max(ns, kkeep) * n, st),
      Cc((size_t)ns * maxsp, st), G((size_t)ns * ns, st), Pm((size_t)ns * ns + 2 * ns + 72, st),
      ework(eig_work_size(maxsp), st);
  SBuf<int> idxbuf((size_t)std::max(nb0, ns) + 8, st);
  int* d_idx = idxbuf.p;
  // Mixed form with eig_fp32: the subspace eigenproblem in FP32 (Ritz
  // residuals of about 1e-7 ||H||, below its tolerance), back to FP64 if the
  // residuals stall.  By default the subspace eigensolve stays FP64.
  bool eig32 = mixed && opt.eig_fp32 && maxsp <= 200;
  bool s32 = false;  // S came from the FP32 solver
  int stall = 0;
  double rprev = 0.0;
  // Ritz vectors X = S V and A X = S (A V) as double-FP32 products in the
  // mixed form (subspace_ff); the orthogonalisation, the restart basis and the
  // projected matrix V^T A V stay FP64
  const bool ffs = mixed && opt.subspace_ff;
  auto sgemm = [&](bool ta, bool tb, int m_, int n_, int k_, double al, const double* A_, int la,
                   const double* B_, int lb, double be, double* C_, int lc) {
    gemm_sub(ffs, ta, tb, m_, n_, k_, al, A_, la, B_, lb, be, C_, lc, st);
  };
  auto product = [&](const double* x, int nv, double* y) {
    if (mixed)
      apply_A_mixed(x, nv, y);
    else
      apply_A_tda(x, nv, y);
  };
  // Preconditioner M = D - s + 2 B^J B^J^T (the orbital-energy differences and
  // the Coulomb part of A, Eq. A_matrix), one shift s below the smallest
  // difference for all states (see CoulPrecond).
  const bool cprec = opt.precond == 0 && nJ > 0;
  CoulPrecond cp;
  if (cprec) cp.setup(*this, true, 2.0, ns);
  auto precondition = [&](int nt) {  // T[j] = M^-1 R[d_idx[j]]
    if (!cprec) {
      k_precond<<<cdiv(n * nt, 256), 256, 0, st>>>(Rr.p, de.p, w.p, d_idx, n, nt, T.p);
      RIS_CHECK_LAUNCH();
      return;
    }
    cp.apply(*this, Rr.p, d_idx, nt, T.p);
  };
  int m = nb0;
  if (guess) {
    // the given rows, optionally followed by unit vectors on the lowest
    // orbital-energy differences, orthonormalised by two CholQR passes that
    // drop rows dependent on earlier ones (the given rows come first)
    const int nunit = augment ? std::max(0, nb0 - nguess) : 0;
    m = nguess + nunit;
    RIS_REQUIRE(m <= 64 && m <= maxsp, RIS_ERR_ARG, "initial Davidson block too large");
    RIS_CUDA(cudaMemcpyAsync(V.p, guess, sizeof(double) * nguess * n, cudaMemcpyDeviceToDevice, st));
    if (nunit > 0) {
      k_lowest<<<1, 1024, 0, st>>>(de.p, (int)n, nunit, d_idx);
      RIS_CHECK_LAUNCH();
      k_unit_rows<<<nunit, 256, 0, st>>>(d_idx, nunit, n, V.p + (size_t)nguess * n);
      RIS_CHECK_LAUNCH();
    }
    SBuf<double> G0((size_t)m * m, st), P0((size_t)m * m + 64, st), W0((size_t)m * m + m, st);
    for (int pass = 0; pass < 2; pass++) {
      row_norms(V.p, m, n, G0.p, st);
      k_scale_rows<<<cdiv(n * m, 256), 256, 0, st>>>(V.p, n, m, G0.p);
      RIS_CHECK_LAUNCH();
      dgemm(false, true, m, m, (int)n, 1.0, V.p, (int)n, V.p, (int)n, 0.0, G0.p, m, st);
      cholqr_small(G0.p, m, 1e-10, P0.p, (int*)(P0.p + m * m), st);
      int nk2 = 0;
      RIS_CUDA(cudaMemcpyAsync(&nk2, P0.p + m * m, sizeof(int), cudaMemcpyDeviceToHost, st));
      RIS_CUDA(cudaStreamSynchronize(st));
      RIS_REQUIRE(nk2 >= ns && (augment || nk2 == m), RIS_ERR_ARG,
                  "initial Davidson block is linearly dependent");
      dgemm(false, false, nk2, (int)n, m, 1.0, P0.p, m, V.p, (int)n, 0.0, tmp.p, (int)n, st);
      RIS_CUDA(cudaMemcpyAsync(V.p, tmp.p, sizeof(double) * nk2 * n, cudaMemcpyDeviceToDevice, st));
      m = nk2;
    }
  } else {
    k_lowest<<<1, 1024, 0, st>>>(de.p, (int)n, nb0, d_idx);
    RIS_CHECK_LAUNCH();
    k_unit_rows<<<nb0, 256, 0, st>>>(d_idx, nb0, n, V.p);
    RIS_CHECK_LAUNCH();
  }
  product(V.p, m, AV.p);
  int nprod = m;
  dgemm(false, true, m, m, (int)n, 1.0, V.p, (int)n, AV.p, (int)n, 0.0, Hs.p, maxsp, st);
  std::vector<double> rn(ns);
  std::vector<double> rhist;
  bool converged = false;
  int it = 0;
  double rmax = 0.0;
  const double drop = 1e-10;
  for (it = 0; it < opt.max_iter; it++) {
    const int nk = std::min(m, std::max(ns, kkeep));
    s32 = eig32 && sym_eig_lowest_f32(Hs.p, maxsp, m, nk, w.p, S.p, ework.p, st);
    if (!s32) sym_eig_lowest(Hs.p, maxsp, m, nk, w.p, S.p, ework.p, st);
    sgemm(false, false, ns, (int)n, m, 1.0, S.p, m, V.p, (int)n, 0.0, Xr.p, (int)n);
    sgemm(false, false, ns, (int)n, m, 1.0, S.p, m, AV.p, (int)n, 0.0, AXr.p, (int)n);
    k_residual<<<cdiv(n * ns, 256), 256, 0, st>>>(AXr.p, Xr.p, w.p, n, ns, Rr.p);
    RIS_CHECK_LAUNCH();
    row_norms(Rr.p, ns, n, G.p, st);
    RIS_CUDA(cudaMemcpyAsync(rn.data(), G.p, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
    RIS_CUDA(cudaStreamSynchronize(st));
    std::vector<int> u;
    rmax = 0.0;
    for (int k = 0; k < ns; k++) {
      if (!(sqrt(rn[k]) <= tol)) u.push_back(k);
      rmax = std::max(rmax, sqrt(rn[k]));
    }
    if (u.empty()) {
      converged = true;
      break;
    }
    if (s32) {  // three iterations without a 10% drop of the largest residual
      stall = it > 0 && rmax > 0.9 * rprev ? stall + 1 : 0;
      if (stall >= 3) eig32 = false;
    }
    rprev = rmax;
    // mixed products: their rounding floor can lie just above the tolerance;
    // eight iterations without a 10% drop of the largest residual, within
    // 100x the tolerance, end the 3xTF32 phase (the caller finishes in FP64)
    rhist.push_back(rmax);
    if (ok && mixed && rhist.size() > 8 && rmax < 100.0 * tol &&
        rmax > 0.9 * rhist[rhist.size() - 9])
      break;
    int nt = (int)u.size();
    RIS_CUDA(cudaMemcpyAsync(d_idx, u.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, st));
    precondition(nt);
    if (m + nt > maxsp) {  // restart with the lowest Ritz vectors
      int keep = std::min(nk, maxsp - nt);
      const double* Sk = S.p;
      SBuf<double> S2(s32 ? (size_t)keep * m : 1, st), T1(s32 ? (size_t)keep * m : 1, st),
          G2(s32 ? (size_t)keep * keep + 64 : 1, st), P2(s32 ? (size_t)keep * keep + 64 : 1, st);
      if (s32) {
        // FP32 Ritz vectors are orthogonal only to FP32 level: orthonormalise
        // them in FP64 (CholQR) and project H on them instead of taking diag(w)
        dgemm(false, true, keep, keep, m, 1.0, S.p, m, S.p, m, 0.0, G2.p, keep, st);
        cholqr_small(G2.p, keep, 1e-10, P2.p, (int*)(P2.p + keep * keep), st);
        int nk2 = 0;
        RIS_CUDA(cudaMemcpyAsync(&nk2, P2.p + keep * keep, sizeof(int), cudaMemcpyDeviceToHost, st));
        RIS_CUDA(cudaStreamSynchronize(st));
        RIS_REQUIRE(nk2 >= ns, RIS_ERR_NOT_CONVERGED, "Davidson restart lost Ritz vectors");
        keep = nk2;
        dgemm(false, false, keep, m, keep, 1.0, P2.p, keep, S.p, m, 0.0, S2.p, m, st);
        dgemm(false, false, keep, m, m, 1.0, S2.p, m, Hs.p, maxsp, 0.0, T1.p, m, st);
        dgemm(false, true, keep, keep, m, 1.0, T1.p, m, S2.p, m, 0.0, G2.p, keep, st);
        Sk = S2.p;
      }
      dgemm(false, false, keep, (int)n, m, 1.0, Sk, m, V.p, (int)n, 0.0, tmp.p, (int)n, st);
      RIS_CUDA(cudaMemcpyAsync(V.p, tmp.p, sizeof(double) * keep * n, cudaMemcpyDeviceToDevice, st));
      dgemm(false, false, keep, (int)n, m, 1.0, Sk, m, AV.p, (int)n, 0.0, tmp.p, (int)n, st);
      RIS_CUDA(cudaMemcpyAsync(AV.p, tmp.p, sizeof(double) * keep * n, cudaMemcpyDeviceToDevice, st));
      if (s32) {
        RIS_CUDA(cudaMemcpy2DAsync(Hs.p, sizeof(double) * maxsp, G2.p, sizeof(double) * keep,
                                   sizeof(double) * keep, keep, cudaMemcpyDeviceToDevice, st));
      } else {
        k_diag_set<<<cdiv(keep * keep, 256), 256, 0, st>>>(Hs.p, maxsp, keep, w.p);
        RIS_CHECK_LAUNCH();
      }
      m = keep;
    }
    // up to two rounds of (project out V, orthonormalise within the block).
    // The mixed phase stops after the first when it lost little (every
    // vector keeps at least half its norm under the projection, no vector
    // dropped, smallest CholQR pivot >= 1e-4 of its diagonal): then the
    // vectors are orthogonal to V and to each other to ~1e-14, far below its
    // 1e-6 tolerance ("twice is enough" with the test of Daniel, Gragg,
    // Kaufman and Stewart).  The FP64 form always takes both.
    int nkeep = nt;
    // info block: [0] nkeep (int), [1] smallest pivot, [2, 2 + ns) squared
    // norms before the projection, [2 + ns, 2 + 2 ns) after it
    double* info = Pm.p + (size_t)ns * ns + 8;
    std::vector<double> hinfo(2 + 2 * (size_t)ns);
    row_norms(T.p, nt, n, info + 2, st);
    for (int pass = 0; pass < 2 && nkeep > 0; pass++) {
      dgemm(false, true, nt, m, (int)n, 1.0, T.p, (int)n, V.p, (int)n, 0.0, Cc.p, m, st);
      dgemm(false, false, nt, (int)n, m, -1.0, Cc.p, m, V.p, (int)n, 1.0, T.p, (int)n, st);
      row_norms(T.p, nt, n, info + 2 + ns, st);
      k_scale_rows<<<cdiv(n * nt, 256), 256, 0, st>>>(T.p, n, nt, info + 2 + ns);
      RIS_CHECK_LAUNCH();
      dgemm(false, true, nt, nt, (int)n, 1.0, T.p, (int)n, T.p, (int)n, 0.0, G.p, nt, st);
      cholqr_small(G.p, nt, drop, Pm.p, (int*)info, st, info + 1);
      RIS_CUDA(cudaMemcpyAsync(hinfo.data(), info, sizeof(double) * (2 + 2 * (size_t)ns),
                               cudaMemcpyDeviceToHost, st));
      RIS_CUDA(cudaStreamSynchronize(st));
      memcpy(&nkeep, hinfo.data(), sizeof(int));
      if (nkeep == 0) break;
      bool one_pass = mixed && pass == 0 && nkeep == nt && hinfo[1] >= 1e-4;
      for (int j = 0; j < nt && one_pass; j++) one_pass = hinfo[2 + ns + j] >= 0.25 * hinfo[2 + j];
      dgemm(false, false, nkeep, (int)n, nt, 1.0, Pm.p, nt, T.p, (int)n, 0.0, tmp.p, (int)n, st);
      RIS_CUDA(cudaMemcpyAsync(T.p, tmp.p, sizeof(double) * nkeep * n, cudaMemcpyDeviceToDevice, st));
      nt = nkeep;
      if (one_pass) break;
    }
    if (nkeep == 0) break;
    RIS_CUDA(cudaMemcpyAsync(V.p + (size_t)m * n, T.p, sizeof(double) * nt * n,
                             cudaMemcpyDeviceToDevice, st));
    product(T.p, nt, AV.p + (size_t)m * n);
    nprod += nt;
    dgemm(false, true, nt, m + nt, (int)n, 1.0, V.p + (size_t)m * n, (int)n, AV.p, (int)n, 0.0,
          Hs.p + (size_t)m * maxsp, maxsp, st);
    k_mirror<<<cdiv((long long)nt * m + 1, 256), 256, 0, st>>>(Hs.p, maxsp, m, m + nt);
    RIS_CHECK_LAUNCH();
    m += nt;
  }
  stats[4] = nprod;
  stats[5] = it;
  stats[7] = rmax;
  if (ok) *ok = converged;
  RIS_REQUIRE(converged || ok, RIS_ERR_NOT_CONVERGED,
              "Davidson did not converge in " + std::to_string(it) + " iterations (largest residual " +
                  std::to_string(rmax) + ")");
  k_phase<<<ns, 256, 0, st>>>(Xr.p, nullptr, n);
  RIS_CHECK_LAUNCH();
  nstates = ns;
  omega.ensure(ns, st);
  X.ensure((size_t)ns * n, st);
  RIS_CUDA(cudaMemcpyAsync(omega.p, w.p, sizeof(double) * ns, cudaMemcpyDeviceToDevice, st));
  RIS_CUDA(cudaMemcpyAsync(X.p, Xr.p, sizeof(double) * ns * n, cudaMemcpyDeviceToDevice, st));
}

void Engine::excite(int ns, double* om, double* Xo, double* Yo, const double* guess) {
  RIS_REQUIRE(stage >= 2, RIS_ERR_STATE, "ris_excite before ris_build_B");
  const long long n = (long long)nocc * nvir;
  RIS_REQUIRE(ns >= 1 && ns <= 32 && ns <= n, RIS_ERR_ARG, "nstates out of range (1..32)");
  RIS_REQUIRE(om, RIS_ERR_ARG, "omega is NULL");
  stage = 2;
  if (opt.rpa) {
    davidson_rpa(ns);
  } else if (guess) {
    SBuf<double> g((size_t)ns * n, st);
    copy_in(g.p, guess, (size_t)ns * n, st);
    davidson_tda(ns, g.p);
  } else {
    davidson_tda(ns);
  }
  h_omega.resize(ns);
  RIS_CUDA(cudaMemcpyAsync(h_omega.data(), omega.p, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
  copy_out(om, omega.p, ns, st);
  if (Xo) copy_out(Xo, X.p, (size_t)ns * n, st);
  if (Yo && opt.rpa) copy_out(Yo, Y.p, (size_t)ns * n, st);
  RIS_CUDA(cudaStreamSynchronize(st));
  stage = 3;
}

// copy the leading m x m block of a matrix with leading dimension ld
__global__ void k_copy_sub(const double* __restrict__ src, int ld, int m, double* __restrict__ dst) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * m) return;
  dst[t] = src[(size_t)(t / m) * ld + t % m];
}
// w2[k] -> omega[k] = sqrt(w2[k]); rows of Y scaled by omega^-1/2
__global__ void k_rpa_omega(const double* __restrict__ w2, int ns, double* __restrict__ om,
                            double* __restrict__ Y, int m) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ns * m) return;
  const int k = t / m;
  const double o = sqrt(fmax(w2[k], 0.0));
  if (t % m == 0) om[k] = o;
  Y[t] *= 1.0 / sqrt(o);
}
// out[k][i] = a * X[k][i] * s[k]^p + b * Y[k][i]   (row scales)
__global__ void k_rowcomb(const double* __restrict__ X, const double* __restrict__ Y,
                          const double* __restrict__ s, double a, double b, int pw, long long n,
                          int nrow, double* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nrow) return;
  const int k = (int)(t / n);
  double f = a;
  if (pw == 1) f *= s[k];
  if (pw == -1) f /= s[k];
  out[t] = f * X[t] + (Y ? b * Y[t] : 0.0);
}

// Davidson for the Casida problem, Eq. (casida), in the symmetric form: with
// a basis V, a+ = V (A+B) V^T and a- = V (A-B) V^T = L L^T, the reduced
// problem (L^T a+ L) y = omega^2 y gives R = X+Y = V^T L y / sqrt(omega) and
// X-Y = a+ R / omega, normalised so that sum X^2 - Y^2 = 1.
void Engine::davidson_rpa(int ns) {
  const bool mixed = opt.precision == RIS_MIXED;
  const double tol = mixed ? std::max(opt.conv_tol, opt.mixed_tol) : opt.conv_tol;
  const long long n = (long long)nocc * nvir;
  const int nb0 = (int)std::min<long long>(n, ns + std::min(ns, 8));
  int maxsp = opt.max_subspace > 0 ? opt.max_subspace : std::max(nb0 + 4 * ns, 10 * ns);
  maxsp = (int)std::min<long long>(std::min(maxsp, 256), n);
  RIS_REQUIRE(maxsp >= std::max(nb0, 2 * ns) + 2, RIS_ERR_ARG, "max_subspace too small for RPA");
  const int ntmax = 2 * ns;
  SBuf<double> V((size_t)maxsp * n, st), PV((size_t)maxsp * n, st), MV((size_t)maxsp * n, st),
      Ap((size_t)maxsp * maxsp, st), Am((size_t)maxsp * maxsp, st), Lc((size_t)maxsp * maxsp, st),
      Ht((size_t)maxsp * maxsp, st), Hm((size_t)maxsp * maxsp, st), S((size_t)64 * maxsp, st),
      w2(64, st), om(64, st), Rs((size_t)ns * maxsp, st), Ls((size_t)ns * maxsp, st),
      Rf((size_t)ns * n, st), Lf((size_t)ns * n, st), rR((size_t)ns * n, st), rL((size_t)ns * n, st),
      T((size_t)ntmax * n, st), tmp((size_t)std::max(ntmax, nb0) * n, st),
      Cc((size_t)ntmax * maxsp + ntmax * ntmax + 64, st), G((size_t)ntmax * ntmax + ntmax, st),
      Pm((size_t)ntmax * ntmax + 64, st), nrm((size_t)2 * ns, st), ework(eig_work_size(maxsp), st);
  SBuf<int> idxbuf((size_t)std::max(nb0, ns) + 8, st);
  int* d_idx = idxbuf.p;
  int nprod = 0;
  auto products = [&](const double* x, int nv, double* p, double* mm) {
    apply_ApB_AmB(x, nv, p, mm);
    nprod += nv;
  };
  // orthonormalise rows [0, nt) of T against V[0, m) and among themselves
  auto orthonormalise = [&](int nt, int m) -> int {
    int nkeep = nt;
    for (int pass = 0; pass < 2 && nkeep > 0; pass++) {
      if (m > 0) {
        dgemm(false, true, nt, m, (int)n, 1.0, T.p, (int)n, V.p, (int)n, 0.0, Cc.p, m, st);
        dgemm(false, false, nt, (int)n, m, -1.0, Cc.p, m, V.p, (int)n, 1.0, T.p, (int)n, st);
      }
      row_norms(T.p, nt, n, G.p, st);
      k_scale_rows<<<cdiv(n * nt, 256), 256, 0, st>>>(T.p, n, nt, G.p);
      RIS_CHECK_LAUNCH();
      dgemm(false, true, nt, nt, (int)n, 1.0, T.p, (int)n, T.p, (int)n, 0.0, G.p, nt, st);
      cholqr_small(G.p, nt, 1e-10, Pm.p, (int*)(Pm.p + nt * nt), st);
      RIS_CUDA(cudaMemcpyAsync(&nkeep, Pm.p + nt * nt, sizeof(int), cudaMemcpyDeviceToHost, st));
      RIS_CUDA(cudaStreamSynchronize(st));
      if (nkeep == 0) break;
      dgemm(false, false, nkeep, (int)n, nt, 1.0, Pm.p, nt, T.p, (int)n, 0.0, tmp.p, (int)n, st);
      RIS_CUDA(cudaMemcpyAsync(T.p, tmp.p, sizeof(double) * nkeep * n, cudaMemcpyDeviceToDevice, st));
      nt = nkeep;
    }
    return nkeep;
  };
  auto subspace_rows = [&](int m0, int m1) {
    // rows m0..m1 of a+ and a-, mirrored
    dgemm(false, true, m1 - m0, m1, (int)n, 1.0, V.p + (size_t)m0 * n, (int)n, PV.p, (int)n, 0.0,
          Ap.p + (size_t)m0 * maxsp, maxsp, st);
    dgemm(false, true, m1 - m0, m1, (int)n, 1.0, V.p + (size_t)m0 * n, (int)n, MV.p, (int)n, 0.0,
          Am.p + (size_t)m0 * maxsp, maxsp, st);
    if (m0 > 0) {
      k_mirror<<<cdiv((long long)(m1 - m0) * m0 + 1, 256), 256, 0, st>>>(Ap.p, maxsp, m0, m1);
      RIS_CHECK_LAUNCH();
      k_mirror<<<cdiv((long long)(m1 - m0) * m0 + 1, 256), 256, 0, st>>>(Am.p, maxsp, m0, m1);
      RIS_CHECK_LAUNCH();
    }
  };
  k_lowest<<<1, 1024, 0, st>>>(de.p, (int)n, nb0, d_idx);
  RIS_CHECK_LAUNCH();
  k_unit_rows<<<nb0, 256, 0, st>>>(d_idx, nb0, n, V.p);
  RIS_CHECK_LAUNCH();
  int m = nb0;
  products(V.p, m, PV.p, MV.p);
  subspace_rows(0, m);
  std::vector<double> rn(2 * ns);
  bool converged = false;
  int it = 0;
  int* d_info = idxbuf.p + std::max(nb0, ns);
  for (it = 0; it < opt.max_iter; it++) {
    // reduced problem
    k_copy_sub<<<cdiv(m * m, 256), 256, 0, st>>>(Am.p, maxsp, m, Lc.p);
    RIS_CHECK_LAUNCH();
    cholesky(Lc.p, m, d_info, st);
    int info = 0;
    RIS_CUDA(cudaMemcpyAsync(&info, d_info, sizeof(int), cudaMemcpyDeviceToHost, st));
    dgemm(false, false, m, m, m, 1.0, Ap.p, maxsp, Lc.p, m, 0.0, Ht.p, m, st);
    dgemm(true, false, m, m, m, 1.0, Lc.p, m, Ht.p, m, 0.0, Hm.p, m, st);
    const int nk = std::min(m, ns);
    sym_eig_lowest(Hm.p, m, m, nk, w2.p, S.p, ework.p, st);
    RIS_CUDA(cudaStreamSynchronize(st));
    RIS_REQUIRE(info == 0, RIS_ERR_ARG, "A-B is not positive definite in the Davidson subspace");
    k_rpa_omega<<<cdiv(ns * m, 256), 256, 0, st>>>(w2.p, ns, om.p, S.p, m);
    RIS_CHECK_LAUNCH();
    // R_sub = y L^T, L_sub = R_sub a+ / omega
    dgemm(false, true, ns, m, m, 1.0, S.p, m, Lc.p, m, 0.0, Rs.p, m, st);
    dgemm(false, false, ns, m, m, 1.0, Rs.p, m, Ap.p, maxsp, 0.0, Ls.p, m, st);
    k_rowcomb<<<cdiv((long long)ns * m, 256), 256, 0, st>>>(Ls.p, nullptr, om.p, 1.0, 0.0, -1, m, ns, Ls.p);
    RIS_CHECK_LAUNCH();
    dgemm(false, false, ns, (int)n, m, 1.0, Rs.p, m, V.p, (int)n, 0.0, Rf.p, (int)n, st);
    dgemm(false, false, ns, (int)n, m, 1.0, Ls.p, m, V.p, (int)n, 0.0, Lf.p, (int)n, st);
    // residuals: (A+B)R - omega L and (A-B)L - omega R
    dgemm(false, false, ns, (int)n, m, 1.0, Rs.p, m, PV.p, (int)n, 0.0, rR.p, (int)n, st);
    dgemm(false, false, ns, (int)n, m, 1.0, Ls.p, m, MV.p, (int)n, 0.0, rL.p, (int)n, st);
    k_rowcomb<<<cdiv(n * ns, 256), 256, 0, st>>>(Lf.p, rR.p, om.p, -1.0, 1.0, 1, n, ns, rR.p);
    RIS_CHECK_LAUNCH();
    k_rowcomb<<<cdiv(n * ns, 256), 256, 0, st>>>(Rf.p, rL.p, om.p, -1.0, 1.0, 1, n, ns, rL.p);
    RIS_CHECK_LAUNCH();
    row_norms(rR.p, ns, n, nrm.p, st);
    row_norms(rL.p, ns, n, nrm.p + ns, st);
    RIS_CUDA(cudaMemcpyAsync(rn.data(), nrm.p, sizeof(double) * 2 * ns, cudaMemcpyDeviceToHost, st));
    RIS_CUDA(cudaStreamSynchronize(st));
    std::vector<int> u;
    for (int k = 0; k < ns; k++)
      if (!(sqrt(rn[k] + rn[ns + k]) <= tol)) u.push_back(k);
    if (u.empty()) {
      converged = true;
      break;
    }
    const int nu = (int)u.size();
    RIS_CUDA(cudaMemcpyAsync(d_idx, u.data(), sizeof(int) * nu, cudaMemcpyHostToDevice, st));
    k_precond<<<cdiv(n * nu, 256), 256, 0, st>>>(rR.p, de.p, om.p, d_idx, n, nu, T.p);
    RIS_CHECK_LAUNCH();
    k_precond<<<cdiv(n * nu, 256), 256, 0, st>>>(rL.p, de.p, om.p, d_idx, n, nu, T.p + (size_t)nu * n);
    RIS_CHECK_LAUNCH();
    int nt = 2 * nu;
    if (m + nt > maxsp) {
      // restart from the current R and L vectors
      RIS_CUDA(cudaMemcpyAsync(tmp.p, T.p, sizeof(double) * nt * n, cudaMemcpyDeviceToDevice, st));
      RIS_CUDA(cudaMemcpyAsync(T.p, Rf.p, sizeof(double) * ns * n, cudaMemcpyDeviceToDevice, st));
      RIS_CUDA(cudaMemcpyAsync(T.p + (size_t)ns * n, Lf.p, sizeof(double) * ns * n,
                               cudaMemcpyDeviceToDevice, st));
      SBuf<double> keepT((size_t)nt * n, st);
      RIS_CUDA(cudaMemcpyAsync(keepT.p, tmp.p, sizeof(double) * nt * n, cudaMemcpyDeviceToDevice, st));
      const int nr = orthonormalise(2 * ns, 0);
      RIS_REQUIRE(nr > 0, RIS_ERR_NOT_CONVERGED, "RPA Davidson restart lost its basis");
      RIS_CUDA(cudaMemcpyAsync(V.p, T.p, sizeof(double) * nr * n, cudaMemcpyDeviceToDevice, st));
      m = nr;
      products(V.p, m, PV.p, MV.p);
      subspace_rows(0, m);
      RIS_CUDA(cudaMemcpyAsync(T.p, keepT.p, sizeof(double) * nt * n, cudaMemcpyDeviceToDevice, st));
      nt = std::min(nt, maxsp - m);
    }
    const int nk2 = orthonormalise(nt, m);
    if (nk2 == 0) break;
    RIS_CUDA(cudaMemcpyAsync(V.p + (size_t)m * n, T.p, sizeof(double) * nk2 * n, cudaMemcpyDeviceToDevice, st));
    products(V.p + (size_t)m * n, nk2, PV.p + (size_t)m * n, MV.p + (size_t)m * n);
    subspace_rows(m, m + nk2);
    m += nk2;
  }
  stats[4] = nprod;
  stats[5] = it;
  RIS_REQUIRE(converged, RIS_ERR_NOT_CONVERGED,
              "RPA Davidson did not converge in " + std::to_string(it) + " iterations");
  nstates = ns;
  omega.ensure(ns, st);
  X.ensure((size_t)ns * n, st);
  Y.ensure((size_t)ns * n, st);
  RIS_CUDA(cudaMemcpyAsync(omega.p, om.p, sizeof(double) * ns, cudaMemcpyDeviceToDevice, st));
  // X = (R + L)/2, Y = (R - L)/2
  k_rowcomb<<<cdiv(n * ns, 256), 256, 0, st>>>(Rf.p, Lf.p, nullptr, 0.5, 0.5, 0, n, ns, X.p);
  RIS_CHECK_LAUNCH();
  k_rowcomb<<<cdiv(n * ns, 256), 256, 0, st>>>(Rf.p, Lf.p, nullptr, 0.5, -0.5, 0, n, ns, Y.p);
  RIS_CHECK_LAUNCH();
  k_phase<<<ns, 256, 0, st>>>(X.p, Y.p, n);
  RIS_CHECK_LAUNCH();
  if (mixed) {
    int h_err = 0;
    RIS_CUDA(cudaMemcpyAsync(&h_err, d_tcerr, sizeof(int), cudaMemcpyDeviceToHost, st));
    RIS_CUDA(cudaStreamSynchronize(st));
    RIS_REQUIRE(h_err == 0, RIS_ERR_TIMEOUT, "a tensor-core GEMM pipeline wait timed out");
  }
}

// ------------------------------------------------------------------ derivatives
// Derivative integrals for the current geometry: FP64 storage, or FP32 in
// mixed precision (the integral recursion itself is FP64 either way).
void Engine::start_D(cudaStream_t s) {
  const size_t plane = (size_t)nao * nao * nU;
  if (opt.precision == RIS_MIXED) {
    D.release();
    Df.ensure(3 * plane, s);
    RIS_CUDA(cudaMemsetAsync(Df.p, 0, sizeof(float) * 3 * plane, s));
    int3c_deriv<float>(ao, aux, pl, xyz.p, Df.p, s);
  } else {
    D.ensure(3 * plane, s);
    RIS_CUDA(cudaMemsetAsync(D.p, 0, sizeof(double) * 3 * plane, s));
    int3c_deriv<double>(ao, aux, pl, xyz.p, D.p, s);
  }
}

// The main stream waits for derivative integrals started on st2; from then
// on the buffer belongs to the main stream (its eventual free is ordered
// after every use there).
void Engine::join_D() {
  if (!D_pending) return;
  RIS_CUDA(cudaStreamWaitEvent(st, evD, 0));
  if (D.p) D.st = st;
  if (Df.p) Df.st = st;
  D_pending = false;
}

void Engine::ensure_D() {
  join_D();
  if (have_D) return;
  start_D(st);
  have_D = true;
}

void Engine::pair_derivs(int npair, const int* pairs, int nx, const double* X_in,
                         const double* Y_in, double* out) {
  RIS_REQUIRE(stage >= 2, RIS_ERR_STATE, "derivatives before ris_build_B");
  RIS_REQUIRE(npair >= 1 && pairs, RIS_ERR_ARG, "no pairs");
  const int o = nocc, v = nvir, nn = nao;
  const long long nov = (long long)o * v;
  const double* Xa;
  const double* Ya = nullptr;
  SBuf<double> xin, yin;
  if (X_in) {
    RIS_REQUIRE(nx >= 1, RIS_ERR_ARG, "nx must be positive with X_in");
    xin.ensure((size_t)nx * nov, st);
    copy_in(xin.p, X_in, (size_t)nx * nov, st);
    Xa = xin.p;
    if (Y_in) {
      yin.ensure((size_t)nx * nov, st);
      copy_in(yin.p, Y_in, (size_t)nx * nov, st);
      Ya = yin.p;
    }
  } else {
    RIS_REQUIRE(stage >= 3, RIS_ERR_STATE, "no amplitudes: call ris_excite or pass X_in");
    nx = nstates;
    Xa = X.p;
    if (opt.rpa) Ya = Y.p;
  }
  for (int g = 0; g < npair; g++)
    for (int q = 0; q < 2; q++)
      RIS_REQUIRE(pairs[2 * g + q] >= 0 && pairs[2 * g + q] < nx, RIS_ERR_ARG,
                  "state index out of range");
  const bool rpa = Ya != nullptr;
  // unique states
  std::vector<int> su;
  std::map<int, int> slot;
  for (int g = 0; g < 2 * npair; g++)
    if (!slot.count(pairs[g])) {
      slot[pairs[g]] = (int)su.size();
      su.push_back(pairs[g]);
    }
  const int nsu = (int)su.size();
  if (streamed) {
    RIS_REQUIRE(!rpa, RIS_ERR_ARG, "the streamed form is TDA only");
    pair_derivs_streamed(npair, pairs, nsu, su, slot, Xa, out);
    return;
  }
  ensure_D();
  // per state: R, L, D^R = C_o R C_v^T, c^J, Q_R = R C_v^T, Q_L = L C_v^T
  SBuf<double> Rs((size_t)nsu * nov, st), Ls((size_t)nsu * nov, st), DR, cJ, QR, QL, t1;
  for (int s = 0; s < nsu; s++) {
    const double* xs = Xa + (size_t)su[s] * nov;
    const double* ys = rpa ? Ya + (size_t)su[s] * nov : nullptr;
    axpby(nov, 1.0, xs, 1.0, ys, Rs.p + s * nov, st);
    axpby(nov, 1.0, xs, -1.0, ys, Ls.p + s * nov, st);
  }
  DR.ensure((size_t)nsu * nn * nn, st);
  t1.ensure((size_t)nn * v, st);
  cJ.ensure((size_t)nsu * nJ, st);
  w5.ensure((size_t)nsu * nJ, st);
  const double* Co = C.p;
  const double* Cv = C.p + o;
  const bool mixed = opt.precision == RIS_MIXED;
  const int lv4 = ld4(v), lo4 = ld4(o), kp = ld4(2 * o);
  // mixed: splits of R and L [s][i][a]; W_R / W_L = [Q^T | C_o] as [s][nu][k']
  SBuf<float> RSh, RSl, LSh, LSl, WRh, WRl, WLh, WLl;
  if (mixed) {
    RSh.ensure((size_t)nsu * o * lv4, st);
    RSl.ensure((size_t)nsu * o * lv4, st);
    LSh.ensure((size_t)nsu * o * lv4, st);
    LSl.ensure((size_t)nsu * o * lv4, st);
    WRh.ensure((size_t)nsu * nn * kp, st, true);
    WRl.ensure((size_t)nsu * nn * kp, st, true);
    WLh.ensure((size_t)nsu * nn * kp, st, true);
    WLl.ensure((size_t)nsu * nn * kp, st, true);
    split_f64(Rs.p, nsu * o, v, v, RSh.p, RSl.p, lv4, st);
    split_f64(Ls.p, nsu * o, v, v, LSh.p, LSl.p, lv4, st);
    // every state in one launch per kind (batch index = state)
    // D^R_s = C_o R_s C_v^T: t1_s = C_o R_s (split), D^R_s = t1_s C_v^T
    SBuf<float> RtH((size_t)nsu * v * lo4, st), RtL((size_t)nsu * v * lo4, st),
        t1H((size_t)nsu * nn * lv4, st), t1L((size_t)nsu * nn * lv4, st);
    split_f64_t(Rs.p, o, v, v, RtH.p, RtL.p, lo4, st, nsu, nov, (long long)v * lo4);
    tcg(nn, v, o, CoH.p, CoL.p, lo4, RtH.p, RtL.p, lo4, (long long)v * lo4, nsu,
        ep_split(t1H.p, t1L.p, lv4, 1, (long long)nn * lv4), d_tcerr, st);
    tcg(nn, nn, v, t1H.p, t1L.p, lv4, CvH.p, CvL.p, lv4, 0, nsu,
        ep_f64(DR.p, nn, (long long)nn * nn), d_tcerr, st, (long long)nn * lv4, nsu);
    // Q^T_s[nu][i] = sum_a C_v[nu][a] U_s[i][a] into W_s[:, 0:o]; C_o into W_s[:, o:2o]
    for (int w = 0; w < (rpa ? 2 : 1); w++) {
      float* Wh = w == 0 ? WRh.p : WLh.p;
      float* Wl = w == 0 ? WRl.p : WLl.p;
      const float* Uh = w == 0 ? RSh.p : LSh.p;
      const float* Ul = w == 0 ? RSl.p : LSl.p;
      tcg(nn, o, v, CvH.p, CvL.p, lv4, Uh, Ul, lv4, (long long)o * lv4, nsu,
          ep_split(Wh, Wl, kp, 1, (long long)nn * kp), d_tcerr, st);
      const dim3 gc(cdiv((long long)nn * o, 256), nsu);
      k_copy_cols<<<gc, 256, 0, st>>>(CoH.p, lo4, Wh, kp, o, nn, o, (long long)nn * kp);
      RIS_CHECK_LAUNCH();
      k_copy_cols<<<gc, 256, 0, st>>>(CoL.p, lo4, Wl, kp, o, nn, o, (long long)nn * kp);
      RIS_CHECK_LAUNCH();
    }
  }
  if (!mixed || rpa) {
    QR.ensure((size_t)nsu * o * nn, st);
    QL.ensure((size_t)nsu * o * nn, st);
    for (int s = 0; s < nsu; s++) {
      if (!mixed) {
        dgemm(false, false, nn, v, o, 1.0, Co, nmo, Rs.p + s * nov, v, 0.0, t1.p, v, st);
        dgemm(false, true, nn, nn, v, 1.0, t1.p, v, Cv, nmo, 0.0, DR.p + (size_t)s * nn * nn, nn, st);
      }
      dgemm(false, true, o, nn, v, 1.0, Rs.p + s * nov, v, Cv, nmo, 0.0, QR.p + (size_t)s * o * nn, nn, st);
      dgemm(false, true, o, nn, v, 1.0, Ls.p + s * nov, v, Cv, nmo, 0.0, QL.p + (size_t)s * o * nn, nn, st);
    }
  }
  // u_s = R_s . B^J (nJ), c_s = u_s L^-1 (row vector)
  dgemm(false, false, nsu, nJ, (int)nov, 1.0, Rs.p, (int)nov, BJ.p, nJ, 0.0, w5.p, nJ, st);
  dgemm(false, false, nsu, nJ, nJ, 1.0, w5.p, nJ, LJinv.p, nJ, 0.0, cJ.p, nJ, st);
  // Coulomb part of every pair density from per-state data: symmetrised
  // D^R and c^J on the union index (the contraction forms G^J on the fly)
  k_symmetrize_sq<<<cdiv((long long)nsu * nn * nn, 256), 256, 0, st>>>(DR.p, nn, nsu);
  RIS_CHECK_LAUNCH();
  SBuf<double> cU((size_t)nsu * nU, st, true);
  k_expand_cJ<<<cdiv(nsu * nJ, 256), 256, 0, st>>>(cJ.p, d_jU, nsu, nJ, nU, cU.p);
  RIS_CHECK_LAUNCH();
  // Coulomb part: Y_s = D . DRs_s for every state, kCBatch states per pass
  SBuf<double> Yst((size_t)nsu * 3 * nn * nU, st);
  prof_begin(kProfContract, st);
  const double dbytes = mixed ? 4.0 : 8.0;  // derivative integrals in FP32 / FP64
  const int nbat = cdiv(nsu, kCBatch);
  const size_t dtb = (size_t)nn * nn * kCBatch;  // one batch of regrouped densities
  SBuf<float> DRf(mixed ? nbat * dtb : 1, st);
  SBuf<double> DRd(mixed ? 1 : nbat * dtb, st);
  if (mixed)
    k_states_t<float><<<dim3(cdiv((long long)nn * nn, 256), nbat), 256, 0, st>>>(DR.p, nsu, nn, DRf.p);
  else
    k_states_t<double><<<dim3(cdiv((long long)nn * nn, 256), nbat), 256, 0, st>>>(DR.p, nsu, nn, DRd.p);
  RIS_CHECK_LAUNCH();
  const int slJ = pick_slices((long long)nn * nU, nbAvg);
  SBuf<double> partJ((size_t)slJ * std::min(nsu, kCBatch) * 3 * nn * nU, st);
  for (int s0 = 0; s0 < nsu; s0 += kCBatch) {
    const int ns = std::min(kCBatch, nsu - s0);
    const dim3 grid(cdiv((long long)nn * nU, 128), slJ);
    const size_t bo = (size_t)(s0 / kCBatch) * dtb;
    if (mixed)
      k_contract_states<float><<<grid, 128, 0, st>>>(Df.p, DRf.p + bo, ns, nn, nU, slJ, nbPtr.p,
                                                     nbCol.p, partJ.p);
    else
      k_contract_states<double><<<grid, 128, 0, st>>>(D.p, DRd.p + bo, ns, nn, nU, slJ, nbPtr.p,
                                                      nbCol.p, partJ.p);
    RIS_CHECK_LAUNCH();
    const long long cnt = (long long)ns * 3 * nn * nU;
    k_sum_slices<<<cdiv(cnt, 256), 256, 0, st>>>(partJ.p, slJ, cnt,
                                                Yst.p + (size_t)s0 * 3 * nn * nU);
    RIS_CHECK_LAUNCH();
  }
  prof_end(kProfContract, st, dbytes * cdiv(nsu, kCBatch) * (3.0 * nn * nn * nU) +
                                  8.0 * (nsu * (double)nn * nn + 3.0 * nsu * nn * nU));
  // exchange part: pairs in batches sharing one pass over the derivative
  // integrals; G^K[mu][nu][P < nK] and Omega are formed per pair
  const int NB = std::min(npair, kCBatch);
  const size_t gk = (size_t)nn * nn * nK;
  // G^K in FP32 when every term of it comes from the tensor cores (mixed TDA)
  const bool gk32 = mixed && !rpa;
  SBuf<double> GK(gk32 ? 1 : (size_t)NB * gk, st), OmB((size_t)NB * nU * nU, st),
      WK((size_t)NB * 3 * nn * nK, st), Z, Goo, M1, WV;
  SBuf<float> GK32(gk32 ? (size_t)NB * gk : 1, st);
  const int slK = pick_slices((long long)nn * nK, nbAvg);
  SBuf<double> partK((size_t)slK * NB * 3 * nn * nK, st);
  SBuf<int> pst(2 * NB, st);
  if (opt.precision != RIS_MIXED) {
    Z.ensure((size_t)o * v * nK, st);
    Goo.ensure((size_t)o * o * nK, st);
    M1.ensure((size_t)nn * 2 * o * nK, st);
    WV.ensure((size_t)nn * 2 * o, st);
  }
  const double cx = opt.cx;
  for (int g0 = 0; g0 < npair; g0 += NB) {
    const int nb = std::min(NB, npair - g0);
    // (in mixed TDA the single exchange GEMM writes every element of G^K)
    if (!gk32) RIS_CUDA(cudaMemsetAsync(GK.p, 0, sizeof(double) * nb * gk, st));
    RIS_CUDA(cudaMemsetAsync(OmB.p, 0, sizeof(double) * nb * nU * nU, st));
    std::vector<int> h_pst(2 * nb);
    for (int b = 0; b < nb; b++) {
      const int g = g0 + b;
      const int sI = slot[pairs[2 * g]], sJ = slot[pairs[2 * g + 1]];
      h_pst[2 * b] = sI;
      h_pst[2 * b + 1] = sJ;
      double* Gam = gk32 ? nullptr : GK.p + (size_t)b * gk;
      float* Gam32 = gk32 ? GK32.p + (size_t)b * gk : nullptr;
      double* Om = OmB.p + (size_t)b * nU * nU;
      k_omega_J<<<cdiv(nJ * nJ, 256), 256, 0, st>>>(cJ.p + (size_t)sI * nJ, cJ.p + (size_t)sJ * nJ,
                                                     d_jU, nJ, nU, 2.0, Om);
      RIS_CHECK_LAUNCH();
      // exchange (ij|ab) for (R_I,R_J) and (L_I,L_J), each with weight -c_x/2;
      // with Y = 0 both combinations coincide, so one pass with -c_x.
      const int ncomb = rpa ? 2 : 1;
      for (int cmb = 0; cmb < ncomb; cmb++) {
        const double f = rpa ? -0.5 * cx : -cx;
        if (mixed) {
          const size_t so = (size_t)o * lv4, sw = (size_t)nn * kp;
          const float* USh = (cmb == 0 ? RSh.p : LSh.p) + sI * so;
          const float* USl = (cmb == 0 ? RSl.p : LSl.p) + sI * so;
          const float* VSh = (cmb == 0 ? RSh.p : LSh.p) + sJ * so;
          const float* VSl = (cmb == 0 ? RSl.p : LSl.p) + sJ * so;
          const float* WUh = (cmb == 0 ? WRh.p : WLh.p) + sI * sw;
          const float* WUl = (cmb == 0 ? WRl.p : WLl.p) + sI * sw;
          const float* WVh = (cmb == 0 ? WRh.p : WLh.p) + sJ * sw;
          const float* WVl = (cmb == 0 ? WRl.p : WLl.p) + sJ * sw;
          gamma_K_mixed(USh, USl, VSh, VSl, WUh, WUl, WVh, WVl, f, Gam, Gam32, Om);
          continue;
        }
        const double* U = (cmb == 0 ? Rs.p : Ls.p) + (size_t)sI * nov;
        const double* Vv = (cmb == 0 ? Rs.p : Ls.p) + (size_t)sJ * nov;
        const double* QU = (cmb == 0 ? QR.p : QL.p) + (size_t)sI * o * nn;
        const double* QV = (cmb == 0 ? QR.p : QL.p) + (size_t)sJ * o * nn;
        // Z[j][b][P] = sum_a U[j][a] c^vv[a][b][P]
        dgemm(false, false, o, v * nK, v, 1.0, U, v, cKvv.p, v * nK, 0.0, Z.p, v * nK, st);
        // G[j][k][P] = sum_b V[k][b] Z[j][b][P]
        {
          GemmBatch bt;
          bt.nb1 = o;
          bt.sB1 = (long long)v * nK;
          bt.sC1 = (long long)o * nK;
          dgemm(false, false, o, nK, v, 1.0, Vv, v, Z.p, nK, 0.0, Goo.p, nK, st, bt);
        }
        // M1[mu][0:o][P] = C_o G ; M1[mu][o:2o][P] = Q_U^T c^oo
        dgemm(false, false, nn, o * nK, o, 1.0, Co, nmo, Goo.p, o * nK, 0.0, M1.p, 2 * o * nK, st);
        dgemm(true, false, nn, o * nK, o, 1.0, QU, nn, cKoo.p, o * nK, 0.0, M1.p + (size_t)o * nK,
              2 * o * nK, st);
        k_build_W<<<cdiv(nn * 2 * o, 256), 256, 0, st>>>(C.p, nmo, QV, nn, o, WV.p);
        RIS_CHECK_LAUNCH();
        // Gamma[mu][nu][P<nK] += f sum_k W_V[nu][k] M1[mu][k][P]
        {
          GemmBatch bt;
          bt.nb1 = nn;
          bt.sB1 = 2LL * o * nK;
          bt.sC1 = (long long)nn * nK;
          dgemm(false, false, nn, nK, 2 * o, f, WV.p, 2 * o, M1.p, nK, 1.0, Gam, nK, st, bt);
        }
        // Omega[P][Q] += f sum_ij c^oo_ij,P G_ij,Q   (K functions are union 0..nK-1)
        dgemm(true, false, nK, nK, o * o, f, cKoo.p, nK, Goo.p, nK, 1.0, Om, nU, st);
      }
      if (rpa) {
        // (ib|ja) terms, weights -c_x/2 for (R_I,R_J) and +c_x/2 for (L_I,L_J):
        //   E1_P = U c_P^T, E2_P = V c_P^T (nocc x nocc), c_P = c^ov[P] as [k][a]
        //   Gamma_ov^T[nu][mu] += w sum_k C_o[nu][k] (E1_P Q_V + E2_P Q_U)[k][mu]
        //   Omega[A][B] += w sum_{k,i} E2_A[k][i] E1_B[i][k]
        SBuf<double> E1((size_t)nK * o * o, st), E2((size_t)nK * o * o, st), E1t((size_t)nK * o * o, st),
            M2((size_t)nK * o * nn, st), M2p((size_t)nK * o * nn, st);
        for (int cmb = 0; cmb < 2; cmb++) {
          const double wgt = cmb == 0 ? -0.5 * cx : 0.5 * cx;
          const double* U = (cmb == 0 ? Rs.p : Ls.p) + (size_t)sI * nov;
          const double* Vv = (cmb == 0 ? Rs.p : Ls.p) + (size_t)sJ * nov;
          const double* QU = (cmb == 0 ? QR.p : QL.p) + (size_t)sI * o * nn;
          const double* QV = (cmb == 0 ? QR.p : QL.p) + (size_t)sJ * o * nn;
          GemmBatch bP;
          bP.nb1 = nK;
          bP.sB1 = nov;
          bP.sC1 = (long long)o * o;
          dgemm(false, true, o, o, v, 1.0, U, v, cKovP.p, v, 0.0, E1.p, o, st, bP);
          dgemm(false, true, o, o, v, 1.0, Vv, v, cKovP.p, v, 0.0, E2.p, o, st, bP);
          GemmBatch bM;
          bM.nb1 = nK;
          bM.sA1 = (long long)o * o;
          bM.sC1 = (long long)o * nn;
          dgemm(false, false, o, nn, o, 1.0, E1.p, o, QV, nn, 0.0, M2.p, nn, st, bM);
          dgemm(false, false, o, nn, o, 1.0, E2.p, o, QU, nn, 1.0, M2.p, nn, st, bM);
          k_permute120<<<cdiv((long long)nK * o * nn, 256), 256, 0, st>>>(M2.p, nK, o, nn, M2p.p);
          RIS_CHECK_LAUNCH();
          GemmBatch bG;
          bG.nb1 = nn;
          bG.sB1 = (long long)nK * o;
          bG.sC1 = (long long)nn * nK;
          dgemm(false, true, nn, nK, o, wgt, C.p, nmo, M2p.p, o, 1.0, Gam, nK, st, bG);
          // E1t[P][k][i] = E1[P][i][k]
          transpose_last2(E1.p, nK, o, o, E1t.p, st);
          dgemm(false, true, nK, nK, o * o, wgt, E2.p, o * o, E1t.p, o * o, 1.0, Om, nU, st);
        }
      }
    }
    RIS_CUDA(cudaMemcpyAsync(pst.p, h_pst.data(), sizeof(int) * 2 * nb, cudaMemcpyHostToDevice, st));
    prof_begin(kProfContract, st);
    const dim3 gridK(cdiv((long long)nn * nK, 128), slK);
    if (gk32)
      k_contract_exchange<float, float><<<gridK, 128, 0, st>>>(Df.p, GK32.p, nb, nn, nU, nK, slK,
                                                              nbPtr.p, nbCol.p, partK.p);
    else if (mixed)
      k_contract_exchange<float, double><<<gridK, 128, 0, st>>>(Df.p, GK.p, nb, nn, nU, nK, slK,
                                                               nbPtr.p, nbCol.p, partK.p);
    else
      k_contract_exchange<double, double><<<gridK, 128, 0, st>>>(D.p, GK.p, nb, nn, nU, nK, slK,
                                                                nbPtr.p, nbCol.p, partK.p);
    RIS_CHECK_LAUNCH();
    const long long cntK = (long long)nb * 3 * nn * nK;
    k_sum_slices<<<cdiv(cntK, 256), 256, 0, st>>>(partK.p, slK, cntK, WK.p);
    RIS_CHECK_LAUNCH();
    // algorithmic bytes: the P < nK part of D once, G^K twice per pair, W written
    prof_end(kProfContract, st,
             dbytes * 3.0 * nn * nn * nK + (gk32 ? 4.0 : 8.0) * 2.0 * nb * gk + 24.0 * nb * nn * nK);
    k_grad_reduce_pairs<<<dim3(natm, nb), 128, 0, st>>>(WK.p, Yst.p, cU.p, pst.p, OmB.p, dMU.p,
                                                        aoPtr.p, aoList.p, axPtr.p, axList.p, nn,
                                                        nU, nK, natm, out + (size_t)g0 * natm * 3);
    RIS_CHECK_LAUNCH();
    RIS_CUDA(cudaStreamSynchronize(st));  // h_pst goes out of scope
  }
  if (opt.precision == RIS_MIXED) {
    int h_err = 0;
    RIS_CUDA(cudaMemcpyAsync(&h_err, d_tcerr, sizeof(int), cudaMemcpyDeviceToHost, st));
    RIS_CUDA(cudaStreamSynchronize(st));
    RIS_REQUIRE(h_err == 0, RIS_ERR_TIMEOUT, "a tensor-core GEMM pipeline wait timed out");
  }
}


// ------------------------------------------------------------------ Z-vector
// (ib|P)_K block B^K_ov as [R][i][a], built on demand when the context was
// not created for RPA (the (A+B) products of the Z-vector need it).
void Engine::ensure_Kov() {
  RIS_REQUIRE(!streamed, RIS_ERR_ARG, "the (ib|P) block is not available in the streamed form");
  const int o = nocc, v = nvir, n = nao;
  const long long nov = (long long)o * v;
  if (BKovR.p && BKovR.n >= (size_t)nov * nK) return;
  RIS_REQUIRE(TK.p, RIS_ERR_STATE, "three-centre integrals not available (trimmed context)");
  const double* Co = C.p;
  const double* Cv = C.p + o;
  SBuf<double> H((size_t)o * n * nK, st), Bia((size_t)nov * nK, st), Bm((size_t)nov * nK, st);
  dgemm(true, false, o, n * nK, n, 1.0, Co, nmo, TK.p, n * nK, 0.0, H.p, n * nK, st);
  GemmBatch bt;
  bt.nb1 = o;
  bt.sB1 = (long long)n * nK;
  bt.sC1 = (long long)v * nK;
  dgemm(true, false, v, nK, n, 1.0, Cv, nmo, H.p, nK, 0.0, Bia.p, nK, st, bt);
  dgemm(false, true, (int)nov, nK, nK, 1.0, Bia.p, nK, LKinv.p, nK, 0.0, Bm.p, nK, st);  // [i][a][R]
  BKovR.ensure((size_t)nov * nK, st);
  transpose_last2(Bm.p, 1, (int)nov, nK, BKovR.p, st);  // [R][ia]
}

// Preconditioned conjugate gradients on (A+B)_ris Z = rhs (Eq. Z_vector with
// the ris kernel of Eq. ris in A+B, the ris-approximated Z-vector solver), all
// right-hand sides at once; preconditioner D + 4 B^J B^J^T (CoulPrecond).
// Converged when |r_j| <= tol |rhs_j| for every j.
void Engine::zvector(int nr, const double* rhs_in, double* Z_out) {
  RIS_REQUIRE(stage >= 2, RIS_ERR_STATE, "ris_zvector before ris_build_B");
  RIS_REQUIRE(nr >= 1 && nr <= 64 && rhs_in && Z_out, RIS_ERR_ARG, "bad Z-vector arguments");
  ensure_Kov();
  const long long n = (long long)nocc * nvir;
  const size_t sz = (size_t)nr * n;
  SBuf<double> b(sz, st), x(sz, st, true), r(sz, st), z(sz, st), p(sz, st), q(sz, st);
  SBuf<double> sc(5 * (size_t)nr, st);  // rz, pq, rzn, |r|^2, |b|^2
  double* rz = sc.p;
  double* pq = sc.p + nr;
  double* rzn = sc.p + 2 * nr;
  double* rr = sc.p + 3 * nr;
  double* bb = sc.p + 4 * nr;
  SBuf<int> act(nr, st);
  copy_in(b.p, rhs_in, sz, st);
  RIS_CUDA(cudaMemcpyAsync(r.p, b.p, sizeof(double) * sz, cudaMemcpyDeviceToDevice, st));
  const bool mixed = opt.precision == RIS_MIXED;
  const double tol = mixed ? std::max(opt.conv_tol, opt.mixed_tol) : opt.conv_tol;
  CoulPrecond cp;
  const bool cprec = nJ > 0;
  auto precondition = [&](const double* R, double* T) {
    if (cprec) {
      cp.apply(*this, R, nullptr, nr, T);
    } else {  // diagonal
      SBuf<double> w0(nr, st, true);
      SBuf<int> idx(nr, st);
      std::vector<int> h(nr);
      for (int j = 0; j < nr; j++) h[j] = j;
      RIS_CUDA(cudaMemcpyAsync(idx.p, h.data(), sizeof(int) * nr, cudaMemcpyHostToDevice, st));
      k_precond<<<cdiv(n * nr, 256), 256, 0, st>>>(R, de.p, w0.p, idx.p, n, nr, T);
      RIS_CHECK_LAUNCH();
      RIS_CUDA(cudaStreamSynchronize(st));
    }
  };
  if (cprec) cp.setup(*this, false, 4.0, nr);
  std::vector<int> h_act(nr, 1);
  std::vector<double> h_rr(nr), h_bb(nr);
  k_row_dots<<<nr, 256, 0, st>>>(b.p, b.p, n, bb);
  RIS_CHECK_LAUNCH();
  RIS_CUDA(cudaMemcpyAsync(h_bb.data(), bb, sizeof(double) * nr, cudaMemcpyDeviceToHost, st));
  precondition(r.p, z.p);
  RIS_CUDA(cudaMemcpyAsync(p.p, z.p, sizeof(double) * sz, cudaMemcpyDeviceToDevice, st));
  k_row_dots<<<nr, 256, 0, st>>>(r.p, z.p, n, rz);
  RIS_CHECK_LAUNCH();
  RIS_CUDA(cudaStreamSynchronize(st));
  for (int j = 0; j < nr; j++) h_act[j] = h_bb[j] > 0.0;
  int it = 0, nprod = 0;
  bool converged = false;
  for (it = 0; it < opt.max_iter; it++) {
    RIS_CUDA(cudaMemcpyAsync(act.p, h_act.data(), sizeof(int) * nr, cudaMemcpyHostToDevice, st));
    apply_ApB_AmB(p.p, nr, q.p, nullptr);
    nprod += nr;
    k_row_dots<<<nr, 256, 0, st>>>(p.p, q.p, n, pq);
    RIS_CHECK_LAUNCH();
    k_cg_xr<<<cdiv(n * nr, 256), 256, 0, st>>>(x.p, r.p, p.p, q.p, rz, pq, act.p, n, nr);
    RIS_CHECK_LAUNCH();
    k_row_dots<<<nr, 256, 0, st>>>(r.p, r.p, n, rr);
    RIS_CHECK_LAUNCH();
    RIS_CUDA(cudaMemcpyAsync(h_rr.data(), rr, sizeof(double) * nr, cudaMemcpyDeviceToHost, st));
    RIS_CUDA(cudaStreamSynchronize(st));
    bool any = false;
    for (int j = 0; j < nr; j++) {
      if (h_act[j] && sqrt(h_rr[j]) <= tol * sqrt(h_bb[j])) h_act[j] = 0;
      any = any || h_act[j];
    }
    if (!any) {
      converged = true;
      break;
    }
    RIS_CUDA(cudaMemcpyAsync(act.p, h_act.data(), sizeof(int) * nr, cudaMemcpyHostToDevice, st));
    precondition(r.p, z.p);
    k_row_dots<<<nr, 256, 0, st>>>(r.p, z.p, n, rzn);
    RIS_CHECK_LAUNCH();
    k_cg_p<<<cdiv(n * nr, 256), 256, 0, st>>>(p.p, z.p, rzn, rz, act.p, n, nr);
    RIS_CHECK_LAUNCH();
    RIS_CUDA(cudaMemcpyAsync(rz, rzn, sizeof(double) * nr, cudaMemcpyDeviceToDevice, st));
  }
  stats[4] = nprod;
  stats[5] = it + 1;
  double worst = 0.0;
  for (int j = 0; j < nr; j++)
    if (h_bb[j] > 0) worst = std::max(worst, sqrt(h_rr[j] / h_bb[j]));
  stats[7] = worst;
  RIS_REQUIRE(converged, RIS_ERR_NOT_CONVERGED,
              "Z-vector CG did not converge in " + std::to_string(it) + " iterations");
  if (opt.precision == RIS_MIXED) {
    int h_err = 0;
    RIS_CUDA(cudaMemcpyAsync(&h_err, d_tcerr, sizeof(int), cudaMemcpyDeviceToHost, st));
    RIS_CUDA(cudaStreamSynchronize(st));
    RIS_REQUIRE(h_err == 0, RIS_ERR_TIMEOUT, "a tensor-core GEMM pipeline wait timed out");
  }
  copy_out(Z_out, x.p, sz, st);
  RIS_CUDA(cudaStreamSynchronize(st));
}


// ------------------------------------------------------------------ streamed form
// For systems whose dense AO three-index tensors do not fit in device memory
// (Sec. 3: the three-centre tensors are batched along the AO or auxiliary
// index, with recomputation):
//   * (mu nu|P) is computed only on the screened function pairs and mixed
//     there with the metric factors, (mu nu|R)_X = sum_P (mu nu|P) (L_X^-1)_RP,
//     so that each MO transform yields final B tensors (no accumulation over
//     auxiliary blocks);
//   * the MO transforms run over blocks of R, each block scattered into a
//     dense [mu][nu][r] buffer;
//   * the exchange part of every Davidson product runs over blocks of
//     occupied orbitals (apply_exchange_mixed);
//   * the gradient regenerates the derivative integrals block by block of
//     auxiliary functions and contracts each block at once; the exchange
//     density is formed from B^K_vv (G~_R = U B_R V^T, then mixed with L_K^-1)
//     so that the fitting coefficients c^K_vv are never stored.

// T[mu][nu][r] = T[nu][mu][r] = Bao[f][r0 + r] for the function pair f = (mu, nu)
__global__ void k_fp_scatter(const double* __restrict__ Bao, int ldB, int r0, int rw, long long nfp,
                             const int* __restrict__ fmu, const int* __restrict__ fnu, int n,
                             double* __restrict__ T) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nfp * rw) return;
  const long long f = t / rw;
  const int r = (int)(t % rw);
  const double x = Bao[(size_t)f * ldB + r0 + r];
  const int mu = fmu[f], nu = fnu[f];
  T[((size_t)mu * n + nu) * rw + r] = x;
  T[((size_t)nu * n + mu) * rw + r] = x;
}

// Lu[R][u] = Linv[R][map[u]] (0 where map[u] < 0), R < nr, u < nu
__global__ void k_gather_metric(const double* __restrict__ Linv, int nr, const int* __restrict__ map,
                                int nu, double* __restrict__ Lu) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nr * nu) return;
  const int R = t / nu, u = t % nu;
  const int j = map[u];
  Lu[t] = j >= 0 ? Linv[(size_t)R * nr + j] : 0.0;
}

// out[b][r0 + r][a] = G[a][b][r] (FP64 B^K_vv in the Davidson layout)
__global__ void k_place_vv(const double* __restrict__ G, int v, int rw, int r0, int nK,
                           double* __restrict__ out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)v * v * rw) return;
  const int r = (int)(t % rw);
  const long long ab = t / rw;
  const int b = (int)(ab % v), a = (int)(ab / v);
  out[((size_t)b * nK + r0 + r) * v + a] = G[t];
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Exact a <-> b symmetry of B^K_vv in its split storage [a][R][b] (row
// length ldb): both elements become their FP64 mean, split again.
__global__ void k_sym_split(float* __restrict__ hi, float* __restrict__ lo, int v, int nK, int ldb) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)v * v * nK) return;
  const int b = (int)(t % v);
  const long long aR = t / v;
  const int R = (int)(aR % nK), a = (int)(aR / nK);
  if (b <= a) return;
  const size_t p = ((size_t)a * nK + R) * ldb + b, q = ((size_t)b * nK + R) * ldb + a;
  const double m = 0.5 * (((double)hi[p] + (double)lo[p]) + ((double)hi[q] + (double)lo[q]));
  const float x = (float)m;
  const float h = tf32_round(x), l = tf32_round(x - h);
  hi[p] = h;
  lo[p] = l;
  hi[q] = h;
  lo[q] = l;
}

// out[row][u0 + c] = sum_s part[s][row][c], row < rows, c < w (fixed order)
__global__ void k_sum_slices_cols(const double* __restrict__ part, int nslice, long long rows, int w,
                                  double* __restrict__ out, int ldo, int u0) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * w) return;
  const long long row = t / w;
  const int c = (int)(t % w);
  double acc = 0.0;
  for (int sl = 0; sl < nslice; sl++) acc += part[(size_t)sl * rows * w + t];
  out[(size_t)row * ldo + u0 + c] = acc;
}

bool Engine::want_streamed(int n) const {
  if (opt.stream > 0) return true;
  if (opt.stream < 0) return false;
  size_t fr = 0, tot = 0;
  RIS_CUDA(cudaMemGetInfo(&fr, &tot));
  const double cap = opt.mem_budget ? (double)opt.mem_budget : (double)tot;
  const double dense = 8.0 * n * n * (double)(nJ + nK) +
                       (opt.precision == RIS_MIXED ? 4.0 : 8.0) * 3.0 * n * n * (double)nU;
  return dense > cap / 3.0;
}

// Functions per block for a buffer of bytes_per_function per function: up to
// 24 GB or 12% of the free device memory (or the stream_block option).
int Engine::block_width(double per) const {
  if (opt.stream_block > 0) return opt.stream_block;
  size_t fr = 0, tot = 0;
  RIS_CUDA(cudaMemGetInfo(&fr, &tot));
  const double room = std::min(24.0e9, 0.12 * (double)fr);
  return (int)std::max(1.0, std::min(256.0, std::floor(room / per)));
}

static void scatter_block(const double* Bao, int ldB, int r0, int rw, long long nfp, const int* fmu,
                          const int* fnu, int n, double* T, cudaStream_t st) {
  RIS_CUDA(cudaMemsetAsync(T, 0, sizeof(double) * (size_t)n * n * rw, st));
  k_fp_scatter<<<(unsigned)cdiv(nfp * rw, 256), 256, 0, st>>>(Bao, ldB, r0, rw, nfp, fmu, fnu, n, T);
  RIS_CHECK_LAUNCH();
}

// After the metric factors: the screened function pairs, (mu nu|P) on them,
// the metric-mixed tensors B^J_AO = (mu nu|P) L_J^-T and B^K_AO (K functions
// are the first nK union functions), and the auxiliary blocks.
void Engine::setup_streamed() {
  const int n = nao;
  const std::vector<int>& ha = h_pa;
  const std::vector<int>& hb = h_pb;
  std::vector<long long> po(std::max(pl.npair, 1), 0);
  std::vector<int> fm, fn;
  long long f = 0;
  for (int ip = 0; ip < pl.npair; ip++) {
    const int sa = ha[ip], sb = hb[ip];
    const int na = ncart(ao.h_l[sa]), nb = ncart(ao.h_l[sb]);
    po[ip] = f;
    for (int ia = 0; ia < na; ia++)
      for (int ib = 0; ib < nb; ib++) {
        fm.push_back(ao.h_off[sa] + ia);
        fn.push_back(ao.h_off[sb] + ib);
      }
    f += na * nb;
  }
  RIS_REQUIRE(f > 0 && f < (1ll << 31), RIS_ERR_ARG, "screened function pairs out of range");
  nfp = f;
  pOff.ensure(po.size(), st);
  fpMu.ensure(fm.size(), st);
  fpNu.ensure(fn.size(), st);
  RIS_CUDA(cudaMemcpyAsync(pOff.p, po.data(), sizeof(long long) * po.size(), cudaMemcpyHostToDevice, st));
  RIS_CUDA(cudaMemcpyAsync(fpMu.p, fm.data(), sizeof(int) * fm.size(), cudaMemcpyHostToDevice, st));
  RIS_CUDA(cudaMemcpyAsync(fpNu.p, fn.data(), sizeof(int) * fn.size(), cudaMemcpyHostToDevice, st));
  {
    SBuf<double> Ts((size_t)nfp * nU, st);
    int3c_pairs(ao, aux, pl, xyz.p, pOff.p, Ts.p, st);
    std::vector<int> uJ(nU, -1);
    for (int j = 0; j < nJ; j++) uJ[h_jU[j]] = j;
    SBuf<int> d_uJ(nU, st);
    RIS_CUDA(cudaMemcpyAsync(d_uJ.p, uJ.data(), sizeof(int) * nU, cudaMemcpyHostToDevice, st));
    SBuf<double> LJu((size_t)nJ * nU, st);
    k_gather_metric<<<cdiv((long long)nJ * nU, 256), 256, 0, st>>>(LJinv.p, nJ, d_uJ.p, nU, LJu.p);
    RIS_CHECK_LAUNCH();
    BJao.ensure((size_t)nfp * nJ, st);
    BKao.ensure((size_t)nfp * nK, st);
    if (opt.precision == RIS_MIXED && opt.emu_f64) {
      EmuEpilogue e;
      e.c64 = BJao.p; e.rs = nJ; e.cs = 1;
      emu_abt((int)nfp, nJ, nU, Ts.p, nU, 1, LJu.p, nU, 1, e);
      EmuEpilogue e2;
      e2.c64 = BKao.p; e2.rs = nK; e2.cs = 1;
      emu_abt((int)nfp, nK, nK, Ts.p, nU, 1, LKinv.p, nK, 1, e2);
    } else {
      dgemm(false, true, (int)nfp, nJ, nU, 1.0, Ts.p, nU, LJu.p, nU, 0.0, BJao.p, nJ, st);
      dgemm(false, true, (int)nfp, nK, nK, 1.0, Ts.p, nU, LKinv.p, nK, 0.0, BKao.p, nK, st);
    }
    RIS_CUDA(cudaStreamSynchronize(st));  // host vectors go out of scope
  }
  // auxiliary blocks: runs of union shells within the K part or within the
  // J-only part, sized for the derivative integrals and a batch of exchange
  // densities of the block
  for (ShellSet& b : auxBlk) free_shells(b, st);
  auxBlk.clear();
  blkU0.clear();
  blkW.clear();
  blkWK.clear();
  const double dsz = opt.precision == RIS_MIXED ? 4.0 : 8.0;
  const int wmax = block_width(dsz * 3.0 * n * n + dsz * kCBatch * n * n);
  int s = 0;
  while (s < aux.n) {
    const int lim = s < nKsh ? nKsh : aux.n;
    int e = s, w = 0;
    while (e < lim && (e == s || w + ncart(aux.h_l[e]) <= wmax)) w += ncart(aux.h_l[e++]);
    std::vector<int> a(aux.h_atom.begin() + s, aux.h_atom.begin() + e);
    std::vector<int> l(aux.h_l.begin() + s, aux.h_l.begin() + e);
    std::vector<double> ex(aux.h_ex.begin() + s, aux.h_ex.begin() + e);
    std::vector<int> jm, km;
    int loc = 0;
    for (int q = s; q < e; q++) {
      jm.push_back(loc);
      km.push_back(-1);
      loc += ncart(aux.h_l[q]);
    }
    ShellSet view;
    make_shells(view, a, l, ex, &jm, &km, st);
    auxBlk.push_back(view);
    blkU0.push_back(aux.h_off[s]);
    blkW.push_back(w);
    blkWK.push_back(s < nKsh ? w : 0);
    s = e;
  }
  RIS_CUDA(cudaStreamSynchronize(st));
}

void Engine::build_B_streamed() {
  const int o = nocc, v = nvir, n = nao;
  const long long nov = (long long)o * v;
  const bool mixed = opt.precision == RIS_MIXED;
  RIS_REQUIRE(!opt.rpa, RIS_ERR_ARG, "the streamed form is TDA only");
  RIS_REQUIRE(!(mixed && opt.refine), RIS_ERR_ARG, "refine is not available in the streamed form");
  const bool emu = mixed && opt.emu_f64;
  const int lo4 = ld4(o), lv4 = ld4(v), ldn = ld4(n);
  const double* Co = C.p;
  const double* Cv = C.p + o;
  SBuf<double> Tb;
  // Coulomb: B^J[i][a][R], R in blocks
  BJ.ensure((size_t)nov * nJ, st);
  {
    const int rb = std::min(nJ, block_width(8.0 * n * n * (emu ? 3.5 : 1.0) + 8.0 * n * o * (emu ? 3.5 : 1.0)));
    Tb.ensure((size_t)n * n * rb, st);
    SBuf<double> H((size_t)o * n * rb, st);
    for (int r0 = 0; r0 < nJ; r0 += rb) {
      const int rw = std::min(rb, nJ - r0);
      scatter_block(BJao.p, nJ, r0, rw, nfp, fpMu.p, fpNu.p, n, Tb.p, st);
      if (emu) {  // H[nu][i][r] = sum_mu T[mu][nu][r] C_mu,i ; B[i][a][r] = sum_nu H C_nu,a
        const long long rT = (long long)n * rw, rH = (long long)o * rw;
        EmuEpilogue e1;
        e1.c64 = H.p; e1.rin = rw; e1.rld = rH; e1.rs = 1; e1.cs = rw;
        emu_abt((int)rT, o, n, Tb.p, 1, rT, C.p, 1, nmo, e1);
        EmuEpilogue e2;
        e2.c64 = BJ.p + r0; e2.rin = rw; e2.rld = (long long)v * nJ; e2.rs = 1; e2.cs = nJ;
        emu_abt((int)rH, v, n, H.p, 1, rH, C.p + o, 1, nmo, e2);
      } else {  // H[i][nu][r], then per i: B[i][a][r0 + r]
        dgemm(true, false, o, n * rw, n, 1.0, Co, nmo, Tb.p, n * rw, 0.0, H.p, n * rw, st);
        GemmBatch bt;
        bt.nb1 = o;
        bt.sB1 = (long long)n * rw;
        bt.sC1 = (long long)v * nJ;
        dgemm(true, false, v, rw, n, 1.0, Cv, nmo, H.p, rw, 0.0, BJ.p + r0, nJ, st, bt);
      }
    }
  }
  // exchange: B^K_oo[i][j][R] and B^K_vv (split [a][R][b] in mixed precision,
  // FP64 [b][R][a] otherwise), R in blocks
  BKoo.ensure((size_t)o * o * nK, st);
  if (mixed) {
    BvvH.ensure((size_t)v * nK * lv4, st);
    BvvL.ensure((size_t)v * nK * lv4, st);
  } else {
    BKvvD.ensure((size_t)v * nK * v, st);
  }
  {
    const int rb = std::min(nK, block_width(mixed ? 8.0 * n * n + 8.0 * (double)n * ldn + 8.0 * v * ldn
                                                  : 8.0 * n * n + 8.0 * n * (double)std::max(o, v) + 8.0 * v * v));
    Tb.ensure((size_t)n * n * rb, st);
    if (mixed) {
      if (!d_tcerr) {
        RIS_ALLOC(cudaMallocAsync((void**)&d_tcerr, sizeof(int), st));
        RIS_CUDA(cudaMemsetAsync(d_tcerr, 0, sizeof(int), st));
      }
      SBuf<float> Th((size_t)rb * n * ldn, st, true), Tl((size_t)rb * n * ldn, st, true);
      SBuf<float> CvTh((size_t)v * ldn, st), CvTl((size_t)v * ldn, st);
      SBuf<float> CoTh((size_t)o * ldn, st), CoTl((size_t)o * ldn, st);
      SBuf<float> Hh((size_t)v * rb * ldn, st), Hl((size_t)v * rb * ldn, st);
      split_f64_t(Cv, n, v, nmo, CvTh.p, CvTl.p, ldn, st);  // [a][mu]
      split_f64_t(Co, n, o, nmo, CoTh.p, CoTl.p, ldn, st);  // [i][mu]
      for (int r0 = 0; r0 < nK; r0 += rb) {
        const int rw = std::min(rb, nK - r0);
        scatter_block(BKao.p, nK, r0, rw, nfp, fpMu.p, fpNu.p, n, Tb.p, st);
        split_f64_tpad(Tb.p, (long long)n * n, rw, n, ldn, Th.p, Tl.p, st);  // [r][mu][nu]
        {  // H[a][r][nu] = sum_mu C_mu,a T[r][mu][nu]
          TcEpilogue e = ep_split(Hh.p, Hl.p, (long long)rw * ldn);
          e.cin = n;
          e.cld = ldn;
          tcg(v, rw * n, n, CvTh.p, CvTl.p, ldn, Th.p, Tl.p, ldn, 0, 1, e, d_tcerr, st);
        }
        {  // B[a][r0 + r][b] = sum_nu H[a][r][nu] C_nu,b
          TcEpilogue e = ep_split(BvvH.p + (size_t)r0 * lv4, BvvL.p + (size_t)r0 * lv4, lv4);
          e.rin = rw;
          e.rld = (long long)nK * lv4;
          tcg(v * rw, v, n, Hh.p, Hl.p, ldn, CvTh.p, CvTl.p, ldn, 0, 1, e, d_tcerr, st);
        }
        {  // the oo block the same way
          TcEpilogue e = ep_split(Hh.p, Hl.p, (long long)rw * ldn);
          e.cin = n;
          e.cld = ldn;
          tcg(o, rw * n, n, CoTh.p, CoTl.p, ldn, Th.p, Tl.p, ldn, 0, 1, e, d_tcerr, st);
        }
        {
          TcEpilogue e = ep_f64(BKoo.p + r0, 1, 0, 1.0, 0.0, nK);
          e.rin = rw;
          e.rld = (long long)o * nK;
          tcg(o * rw, o, n, Hh.p, Hl.p, ldn, CoTh.p, CoTl.p, ldn, 0, 1, e, d_tcerr, st);
        }
      }
      k_sym_split<<<(unsigned)cdiv((long long)v * v * nK, 256), 256, 0, st>>>(BvvH.p, BvvL.p, v, nK, lv4);
      RIS_CHECK_LAUNCH();
    } else {
      SBuf<double> H((size_t)std::max(o, v) * n * rb, st), G((size_t)v * v * rb, st);
      for (int r0 = 0; r0 < nK; r0 += rb) {
        const int rw = std::min(rb, nK - r0);
        scatter_block(BKao.p, nK, r0, rw, nfp, fpMu.p, fpNu.p, n, Tb.p, st);
        dgemm(true, false, o, n * rw, n, 1.0, Co, nmo, Tb.p, n * rw, 0.0, H.p, n * rw, st);
        GemmBatch bt;
        bt.nb1 = o;
        bt.sB1 = (long long)n * rw;
        bt.sC1 = (long long)o * nK;
        dgemm(true, false, o, rw, n, 1.0, Co, nmo, H.p, rw, 0.0, BKoo.p + r0, nK, st, bt);
        dgemm(true, false, v, n * rw, n, 1.0, Cv, nmo, Tb.p, n * rw, 0.0, H.p, n * rw, st);
        GemmBatch b2;
        b2.nb1 = v;
        b2.sB1 = (long long)n * rw;
        b2.sC1 = (long long)v * rw;
        dgemm(true, false, v, rw, n, 1.0, Cv, nmo, H.p, rw, 0.0, G.p, rw, st, b2);
        k_place_vv<<<(unsigned)cdiv((long long)v * v * rw, 256), 256, 0, st>>>(G.p, v, rw, r0, nK, BKvvD.p);
        RIS_CHECK_LAUNCH();
      }
    }
  }
  Tb.release();
  // fitting coefficients of the oo block, c = B L^-1, as [P][i][k]
  cKoo.ensure((size_t)o * o * nK, st);
  dgemm(false, false, o * o, nK, nK, 1.0, BKoo.p, nK, LKinv.p, nK, 0.0, cKoo.p, nK, st);
  cKooP.ensure((size_t)o * o * nK, st);
  transpose_last2(cKoo.p, 1, o * o, nK, cKooP.p, st);
  if (mixed) {  // FP32 hi/lo operands of the products and of the gradient
    BooH.ensure((size_t)o * nK * lo4, st);
    BooL.ensure((size_t)o * nK * lo4, st);
    split_f64_t(BKoo.p, o, nK, nK, BooH.p, BooL.p, lo4, st, o, (long long)o * nK, (long long)nK * lo4);
    cooH.ensure((size_t)nK * o * lo4, st);
    cooL.ensure((size_t)nK * o * lo4, st);
    split_f64(cKooP.p, nK * o, o, o, cooH.p, cooL.p, lo4, st);
    CoH.ensure((size_t)n * lo4, st);
    CoL.ensure((size_t)n * lo4, st);
    split_f64(C.p, n, o, nmo, CoH.p, CoL.p, lo4, st);
    CvH.ensure((size_t)n * lv4, st);
    CvL.ensure((size_t)n * lv4, st);
    split_f64(C.p + o, n, v, nmo, CvH.p, CvL.p, lv4, st);
  }
}

// Gradients / coupling numerators of TDA pair energies, streamed form.
void Engine::pair_derivs_streamed(int npair, const int* pairs, int nsu, const std::vector<int>& su,
                                  const std::map<int, int>& slot, const double* Xa, double* out) {
  const int o = nocc, v = nvir, nn = nao;
  const long long nov = (long long)o * v;
  const bool mixed = opt.precision == RIS_MIXED;
  const int lv4 = ld4(v), lo4 = ld4(o), kp = ld4(2 * o), ldK = ld4(nK);
  const double* Co = C.p;
  const double* Cv = C.p + o;
  const double f = -opt.cx;  // TDA: one exchange combination with weight -c_x
  // per state: R = X, D^R = C_o R C_v^T (symmetrised), c^J on the union index
  SBuf<double> Rs((size_t)nsu * nov, st), DR((size_t)nsu * nn * nn, st), cJ((size_t)nsu * nJ, st),
      QR, t1;
  for (int s = 0; s < nsu; s++)
    RIS_CUDA(cudaMemcpyAsync(Rs.p + s * nov, Xa + (size_t)su[s] * nov, sizeof(double) * nov,
                             cudaMemcpyDeviceToDevice, st));
  SBuf<float> RSh, RSl, WRh, WRl, DRf;
  if (mixed) {
    RSh.ensure((size_t)nsu * o * lv4, st);
    RSl.ensure((size_t)nsu * o * lv4, st);
    WRh.ensure((size_t)nsu * nn * kp, st, true);
    WRl.ensure((size_t)nsu * nn * kp, st, true);
    split_f64(Rs.p, nsu * o, v, v, RSh.p, RSl.p, lv4, st);
    SBuf<float> RtH((size_t)nsu * v * lo4, st), RtL((size_t)nsu * v * lo4, st),
        t1H((size_t)nsu * nn * lv4, st), t1L((size_t)nsu * nn * lv4, st);
    split_f64_t(Rs.p, o, v, v, RtH.p, RtL.p, lo4, st, nsu, nov, (long long)v * lo4);
    tcg(nn, v, o, CoH.p, CoL.p, lo4, RtH.p, RtL.p, lo4, (long long)v * lo4, nsu,
        ep_split(t1H.p, t1L.p, lv4, 1, (long long)nn * lv4), d_tcerr, st);
    tcg(nn, nn, v, t1H.p, t1L.p, lv4, CvH.p, CvL.p, lv4, 0, nsu,
        ep_f64(DR.p, nn, (long long)nn * nn), d_tcerr, st, (long long)nn * lv4, nsu);
    // W_R = [Q^T | C_o] as [s][nu][k']
    tcg(nn, o, v, CvH.p, CvL.p, lv4, RSh.p, RSl.p, lv4, (long long)o * lv4, nsu,
        ep_split(WRh.p, WRl.p, kp, 1, (long long)nn * kp), d_tcerr, st);
    const dim3 gc(cdiv((long long)nn * o, 256), nsu);
    k_copy_cols<<<gc, 256, 0, st>>>(CoH.p, lo4, WRh.p, kp, o, nn, o, (long long)nn * kp);
    RIS_CHECK_LAUNCH();
    k_copy_cols<<<gc, 256, 0, st>>>(CoL.p, lo4, WRl.p, kp, o, nn, o, (long long)nn * kp);
    RIS_CHECK_LAUNCH();
  } else {
    QR.ensure((size_t)nsu * o * nn, st);
    t1.ensure((size_t)nn * v, st);
    for (int s = 0; s < nsu; s++) {
      dgemm(false, false, nn, v, o, 1.0, Co, nmo, Rs.p + s * nov, v, 0.0, t1.p, v, st);
      dgemm(false, true, nn, nn, v, 1.0, t1.p, v, Cv, nmo, 0.0, DR.p + (size_t)s * nn * nn, nn, st);
      dgemm(false, true, o, nn, v, 1.0, Rs.p + s * nov, v, Cv, nmo, 0.0, QR.p + (size_t)s * o * nn, nn, st);
    }
  }
  w5.ensure((size_t)nsu * nJ, st);
  dgemm(false, false, nsu, nJ, (int)nov, 1.0, Rs.p, (int)nov, BJ.p, nJ, 0.0, w5.p, nJ, st);
  dgemm(false, false, nsu, nJ, nJ, 1.0, w5.p, nJ, LJinv.p, nJ, 0.0, cJ.p, nJ, st);
  k_symmetrize_sq<<<cdiv((long long)nsu * nn * nn, 256), 256, 0, st>>>(DR.p, nn, nsu);
  RIS_CHECK_LAUNCH();
  // state densities regrouped [batch][mu][nu][b] for the contraction
  const int nbat = cdiv(nsu, kCBatch);
  const size_t dtb = (size_t)nn * nn * kCBatch;
  SBuf<double> DRd(mixed ? 1 : nbat * dtb, st);
  if (mixed) {
    DRf.ensure(nbat * dtb, st);
    k_states_t<float><<<dim3(cdiv((long long)nn * nn, 256), nbat), 256, 0, st>>>(DR.p, nsu, nn, DRf.p);
  } else {
    k_states_t<double><<<dim3(cdiv((long long)nn * nn, 256), nbat), 256, 0, st>>>(DR.p, nsu, nn, DRd.p);
  }
  RIS_CHECK_LAUNCH();
  SBuf<double> cU((size_t)nsu * nU, st, true);
  k_expand_cJ<<<cdiv(nsu * nJ, 256), 256, 0, st>>>(cJ.p, d_jU, nsu, nJ, nU, cU.p);
  RIS_CHECK_LAUNCH();
  SBuf<double> Yst((size_t)nsu * 3 * nn * nU, st);
  // L_K^-T split (mixed): [P][R]
  SBuf<float> LiTh, LiTl;
  if (mixed) {
    LiTh.ensure((size_t)nK * ldK, st, true);
    LiTl.ensure((size_t)nK * ldK, st, true);
    split_f64_t(LKinv.p, nK, nK, nK, LiTh.p, LiTl.p, ldK, st);
  }
  const int NB = std::min(npair, kCBatch);
  int wmaxU = 1, wmaxK = 1;
  for (size_t k = 0; k < blkW.size(); k++) {
    wmaxU = std::max(wmaxU, blkW[k]);
    wmaxK = std::max(wmaxK, blkWK[k]);
  }
  const size_t nn2 = (size_t)nn * nn;
  // per pair of the batch: G[P][k][j] (mixed: split, j padded), Omega
  SBuf<double> Gd(mixed ? 1 : (size_t)NB * nK * o * o, st), OmB((size_t)NB * nU * nU, st),
      WK((size_t)NB * 3 * nn * nK, st);
  SBuf<float> GH(mixed ? (size_t)NB * nK * o * lo4 : 1, st), GL(mixed ? (size_t)NB * nK * o * lo4 : 1, st);
  SBuf<double> D64(mixed ? 1 : 3 * nn2 * wmaxU, st), Gam64(mixed ? 1 : (size_t)NB * nn2 * wmaxK, st);
  SBuf<float> D32(mixed ? 3 * nn2 * wmaxU : 1, st), Gam32(mixed ? (size_t)NB * nn2 * wmaxK : 1, st);
  SBuf<double> M1d(mixed ? 1 : (size_t)nn * wmaxK * 2 * o, st), WVd(mixed ? 1 : (size_t)nn * 2 * o, st);
  SBuf<float> M1h(mixed ? (size_t)nn * wmaxK * kp : 1, st), M1l(mixed ? (size_t)nn * wmaxK * kp : 1, st);
  SBuf<int> pst(2 * NB, st);
  const int slJ = pick_slices((long long)nn * wmaxU, nbAvg), slK = pick_slices((long long)nn * wmaxK, nbAvg);
  SBuf<double> partJ((size_t)slJ * std::min(nsu, kCBatch) * 3 * nn * wmaxU, st),
      partK((size_t)slK * NB * 3 * nn * wmaxK, st);
  const double dbytes = mixed ? 4.0 : 8.0;
  for (int g0 = 0; g0 < npair; g0 += NB) {
    const int nb = std::min(NB, npair - g0);
    RIS_CUDA(cudaMemsetAsync(OmB.p, 0, sizeof(double) * nb * nU * nU, st));
    std::vector<int> h_pst(2 * nb);
    for (int b = 0; b < nb; b++) {
      const int g = g0 + b;
      const int sI = slot.at(pairs[2 * g]), sJ = slot.at(pairs[2 * g + 1]);
      h_pst[2 * b] = sI;
      h_pst[2 * b + 1] = sJ;
      double* Om = OmB.p + (size_t)b * nU * nU;
      k_omega_J<<<cdiv(nJ * nJ, 256), 256, 0, st>>>(cJ.p + (size_t)sI * nJ, cJ.p + (size_t)sJ * nJ, d_jU,
                                                    nJ, nU, 2.0, Om);
      RIS_CHECK_LAUNCH();
      // G~[k][R][j] = sum_ab V_kb B_ab,R U_ja, then G[P][k][j] = sum_R L^-1_RP G~[k][R][j]
      if (mixed) {
        const float* USh = RSh.p + (size_t)sI * o * lv4;
        const float* USl = RSl.p + (size_t)sI * o * lv4;
        const float* VSh = RSh.p + (size_t)sJ * o * lv4;
        const float* VSl = RSl.p + (size_t)sJ * o * lv4;
        SBuf<float> T1h((size_t)nK * o * lv4, st, true), T1l((size_t)nK * o * lv4, st, true);
        {  // T1[R][k][a] = sum_b V[k][b] B[a][R][b]
          TcEpilogue e = ep_split(T1h.p, T1l.p, lv4);
          e.cin = nK;
          e.cld = 1;
          e.cs = (long long)o * lv4;
          tcg(o, v * nK, v, VSh, VSl, lv4, BvvH.p, BvvL.p, lv4, 0, 1, e, d_tcerr, st);
        }
        SBuf<float> Gth((size_t)o * o * ldK, st, true), Gtl((size_t)o * o * ldK, st, true);
        {  // G~[(k, j)][R] = sum_a T1[R][k][a] U[j][a]
          TcEpilogue e = ep_split(Gth.p, Gtl.p, (long long)o * ldK, ldK);
          e.rin = o;
          e.rld = 1;
          tcg(nK * o, o, v, T1h.p, T1l.p, lv4, USh, USl, lv4, 0, 1, e, d_tcerr, st);
        }
        {  // G[P][k][j] = sum_R L^-1[R][P] G~[(k, j)][R]
          float* gh = GH.p + (size_t)b * nK * o * lo4;
          float* gl = GL.p + (size_t)b * nK * o * lo4;
          RIS_CUDA(cudaMemsetAsync(gh, 0, sizeof(float) * nK * o * lo4, st));
          RIS_CUDA(cudaMemsetAsync(gl, 0, sizeof(float) * nK * o * lo4, st));
          TcEpilogue e = ep_split(gh, gl, (long long)o * lo4);
          e.cin = o;
          e.cld = lo4;
          tcg(nK, o * o, nK, LiTh.p, LiTl.p, ldK, Gth.p, Gtl.p, ldK, 0, 1, e, d_tcerr, st);
          // Omega[A][B] += f sum_{k,j} c^oo[A][k][j] G[B][k][j]
          tcg(nK, nK, o * lo4, cooH.p, cooL.p, o * lo4, gh, gl, o * lo4, 0, 1, ep_f64(Om, nU, 0, f, 1.0),
              d_tcerr, st);
        }
      } else {
        const double* U = Rs.p + (size_t)sI * nov;
        const double* V = Rs.p + (size_t)sJ * nov;
        SBuf<double> T1((size_t)o * nK * v, st), Gt((size_t)o * nK * o, st);
        dgemm(false, false, o, nK * v, v, 1.0, V, v, BKvvD.p, nK * v, 0.0, T1.p, nK * v, st);  // [k][R][a]
        dgemm(false, true, o * nK, o, v, 1.0, T1.p, v, U, v, 0.0, Gt.p, o, st);                 // [k][R][j]
        double* G = Gd.p + (size_t)b * nK * o * o;
        GemmBatch bt;
        bt.nb1 = o;
        bt.sB1 = (long long)nK * o;
        bt.sC1 = o;
        dgemm(true, false, nK, o, nK, 1.0, LKinv.p, nK, Gt.p, o, 0.0, G, o * o, st, bt);         // [P][k][j]
        dgemm(false, true, nK, nK, o * o, f, cKooP.p, o * o, G, o * o, 1.0, Om, nU, st);
      }
    }
    RIS_CUDA(cudaMemcpyAsync(pst.p, h_pst.data(), sizeof(int) * 2 * nb, cudaMemcpyHostToDevice, st));
    // auxiliary blocks: derivative integrals regenerated and contracted at once
    for (size_t k = 0; k < auxBlk.size(); k++) {
      const int u0 = blkU0[k], w = blkW[k], wK = blkWK[k];
      if (g0 > 0 && wK == 0) continue;  // the Coulomb part is complete after the first batch
      if (mixed) {
        RIS_CUDA(cudaMemsetAsync(D32.p, 0, sizeof(float) * 3 * nn2 * w, st));
        int3c_deriv<float>(ao, auxBlk[k], pl, xyz.p, D32.p, st);
      } else {
        RIS_CUDA(cudaMemsetAsync(D64.p, 0, sizeof(double) * 3 * nn2 * w, st));
        int3c_deriv<double>(ao, auxBlk[k], pl, xyz.p, D64.p, st);
      }
      prof_begin(kProfContract, st);
      double bytes = 0.0;
      if (g0 == 0) {  // Coulomb part: Y_s[x][mu][u0 + p] for every state
        for (int s0 = 0; s0 < nsu; s0 += kCBatch) {
          const int ns = std::min(kCBatch, nsu - s0);
          const dim3 grid(cdiv((long long)nn * w, 128), slJ);
          const size_t bo = (size_t)(s0 / kCBatch) * dtb;
          if (mixed)
            k_contract_states<float><<<grid, 128, 0, st>>>(D32.p, DRf.p + bo, ns, nn, w, slJ, nbPtr.p,
                                                           nbCol.p, partJ.p);
          else
            k_contract_states<double><<<grid, 128, 0, st>>>(D64.p, DRd.p + bo, ns, nn, w, slJ, nbPtr.p,
                                                            nbCol.p, partJ.p);
          RIS_CHECK_LAUNCH();
          const long long rows = (long long)ns * 3 * nn;
          k_sum_slices_cols<<<(unsigned)cdiv(rows * w, 256), 256, 0, st>>>(
              partJ.p, slJ, rows, w, Yst.p + (size_t)s0 * 3 * nn * nU, nU, u0);
          RIS_CHECK_LAUNCH();
          bytes += dbytes * 3.0 * nn2 * w + 8.0 * ns * nn2;
        }
      }
      if (wK > 0) {  // exchange part of each pair's Gamma for P in the block
        for (int b = 0; b < nb; b++) {
          const int g = g0 + b;
          const int sI = slot.at(pairs[2 * g]), sJ = slot.at(pairs[2 * g + 1]);
          if (mixed) {
            const size_t sw = (size_t)nn * kp;
            const float* gh = GH.p + (size_t)b * nK * o * lo4 + (size_t)u0 * o * lo4;
            const float* gl = GL.p + (size_t)b * nK * o * lo4 + (size_t)u0 * o * lo4;
            // M1[mu][p][k'] : k' < o  sum_i Q_U[i][mu] c^oo[P][i][k]
            //                 k' >= o sum_j C_o[mu][j] G[P][k][j]
            TcEpilogue e = ep_split(M1h.p, M1l.p, (long long)wK * kp);
            e.cin = o;
            e.cld = kp;
            tcg(nn, wK * o, o, WRh.p + sI * sw, WRl.p + sI * sw, kp, cooH.p + (size_t)u0 * o * lo4,
                cooL.p + (size_t)u0 * o * lo4, lo4, 0, 1, e, d_tcerr, st);
            e.chi = M1h.p + o;
            e.clo = M1l.p + o;
            tcg(nn, wK * o, o, CoH.p, CoL.p, lo4, gh, gl, lo4, 0, 1, e, d_tcerr, st);
            // Gamma[mu][nu][p] = f sum_k' W_V[nu][k'] M1[mu][p][k']
            TcEpilogue eg;
            eg.mode = kOutF32;
            eg.c32 = Gam32.p + (size_t)b * nn2 * wK;
            eg.alpha = f;
            eg.beta = 0.0;
            eg.rs = wK;
            eg.cin = wK;
            eg.cld = (long long)nn * wK;
            tcg(nn, nn * wK, 2 * o, WRh.p + sJ * sw, WRl.p + sJ * sw, kp, M1h.p, M1l.p, kp, 0, 1, eg,
                d_tcerr, st);
          } else {
            const double* G = Gd.p + (size_t)b * nK * o * o;
            const double* QU = QR.p + (size_t)sI * o * nn;
            const double* QV = QR.p + (size_t)sJ * o * nn;
            // M1[mu][p][k'] : k' < o  sum_j C_o[mu][j] G[P][k][j]
            //                 k' >= o sum_i Q_U[i][mu] c^oo[P][i][k]
            GemmBatch bp;
            bp.nb1 = wK;
            bp.sB1 = (long long)o * o;
            bp.sC1 = 2LL * o;
            dgemm(false, true, nn, o, o, 1.0, Co, nmo, G + (size_t)u0 * o * o, o, 0.0, M1d.p, wK * 2 * o, st, bp);
            dgemm(true, false, nn, o, o, 1.0, QU, nn, cKooP.p + (size_t)u0 * o * o, o, 0.0, M1d.p + o,
                  wK * 2 * o, st, bp);
            k_build_W<<<cdiv(nn * 2 * o, 256), 256, 0, st>>>(C.p, nmo, QV, nn, o, WVd.p);
            RIS_CHECK_LAUNCH();
            GemmBatch bm;
            bm.nb1 = nn;
            bm.sB1 = (long long)wK * 2 * o;
            bm.sC1 = (long long)nn * wK;
            dgemm(false, true, nn, wK, 2 * o, f, WVd.p, 2 * o, M1d.p, 2 * o, 0.0,
                  Gam64.p + (size_t)b * nn2 * wK, wK, st, bm);
          }
        }
        const dim3 gridK(cdiv((long long)nn * wK, 128), slK);
        if (mixed)
          k_contract_exchange<float, float><<<gridK, 128, 0, st>>>(D32.p, Gam32.p, nb, nn, w, wK, slK,
                                                                   nbPtr.p, nbCol.p, partK.p);
        else
          k_contract_exchange<double, double><<<gridK, 128, 0, st>>>(D64.p, Gam64.p, nb, nn, w, wK, slK,
                                                                     nbPtr.p, nbCol.p, partK.p);
        RIS_CHECK_LAUNCH();
        const long long rows = (long long)nb * 3 * nn;
        k_sum_slices_cols<<<(unsigned)cdiv(rows * wK, 256), 256, 0, st>>>(partK.p, slK, rows, wK, WK.p, nK, u0);
        RIS_CHECK_LAUNCH();
        bytes += dbytes * 3.0 * nn2 * wK + dbytes * 2.0 * nb * nn2 * wK;
      }
      prof_end(kProfContract, st, bytes);
    }
    k_grad_reduce_pairs<<<dim3(natm, nb), 128, 0, st>>>(WK.p, Yst.p, cU.p, pst.p, OmB.p, dMU.p, aoPtr.p,
                                                        aoList.p, axPtr.p, axList.p, nn, nU, nK, natm,
                                                        out + (size_t)g0 * natm * 3);
    RIS_CHECK_LAUNCH();
    RIS_CUDA(cudaStreamSynchronize(st));  // h_pst goes out of scope
  }
  if (mixed) {
    int h_err = 0;
    RIS_CUDA(cudaMemcpyAsync(&h_err, d_tcerr, sizeof(int), cudaMemcpyDeviceToHost, st));
    RIS_CUDA(cudaStreamSynchronize(st));
    RIS_REQUIRE(h_err == 0, RIS_ERR_TIMEOUT, "a tensor-core GEMM pipeline wait timed out");
  }
}

// ------------------------------------------------------------------ time couplings
// T[g] = sum_{A,x} d[g][A][x] v[A][x], one block per pair (fixed-order tree sum)
__global__ void __launch_bounds__(256) k_time_coupling(const double* __restrict__ d,
                                                       const double* __restrict__ vel, int n3,
                                                       double* __restrict__ T) {
  __shared__ double red[256];
  const int g = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < n3; i += 256) s += d[(size_t)g * n3 + i] * vel[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) T[g] = red[0];
}

void Engine::time_coupling(int npair, const double* nac, const double* vel, double* T) {
  RIS_REQUIRE(stage >= 1 && natm > 0, RIS_ERR_STATE, "ris_time_coupling before ris_build_aux");
  RIS_REQUIRE(npair >= 1 && nac && vel && T, RIS_ERR_ARG, "bad time-coupling arguments");
  const int n3 = 3 * natm;
  SBuf<double> dd((size_t)npair * n3, st), vv(n3, st), tt(npair, st);
  copy_in(dd.p, nac, (size_t)npair * n3, st);
  copy_in(vv.p, vel, n3, st);
  k_time_coupling<<<npair, 256, 0, st>>>(dd.p, vv.p, n3, tt.p);
  RIS_CHECK_LAUNCH();
  copy_out(T, tt.p, npair, st);
  RIS_CUDA(cudaStreamSynchronize(st));
}

// ------------------------------------------------------------------ phase tracking
// Align the phases of the current states with those of the previous step
// (X_prev, host or device, [ns][nocc][nvir]); optional copies of the aligned
// amplitudes and of the signs (host or device).
void Engine::phase_align(int ns, const double* Xprev_in, int* sign_out, double* Xout) {
  RIS_REQUIRE(stage >= 2 && nstates > 0 && X.p, RIS_ERR_STATE, "ris_phase_align before ris_excite");
  RIS_REQUIRE(ns >= 1 && ns <= nstates && Xprev_in, RIS_ERR_ARG, "bad phase-alignment arguments");
  const long long n = (long long)nocc * nvir;
  SBuf<double> xp((size_t)ns * n, st);
  copy_in(xp.p, Xprev_in, (size_t)ns * n, st);
  SBuf<int> sg(ns, st);
  k_phase_align<<<ns, 256, 0, st>>>(X.p, opt.rpa ? Y.p : nullptr, xp.p, n, sg.p);
  RIS_CHECK_LAUNCH();
  if (sign_out) {
    cudaPointerAttributes a;
    const bool dev = cudaPointerGetAttributes(&a, sign_out) == cudaSuccess &&
                     (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    RIS_CUDA(cudaMemcpyAsync(sign_out, sg.p, sizeof(int) * ns,
                             dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  }
  if (Xout) copy_out(Xout, X.p, (size_t)ns * n, st);
  RIS_CUDA(cudaStreamSynchronize(st));
}

}  // namespace ris
