// Internal interfaces shared by the CUDA translation units of the library.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>

namespace shp {

// ---- programmatic dependent launch ---------------------------------------------------------------
// Every kernel of the library is launched with programmatic stream serialization: the next kernel
// in a stream is scheduled as soon as every block of the current one has exited, before the grid
// has formally completed, so part of its launch latency overlaps the end of the previous kernel.
// Each kernel therefore begins with pdl_begin(): griddepcontrol.wait blocks until the preceding
// grid has completed and its memory operations are visible, so no read or write of a kernel races
// with its predecessor. Only the tensor-core mode product and its staging copy trigger their
// dependents early (pdl_trigger); elsewhere blocks of a waiting grid would hold warp slots and
// shared memory that a concurrent stream's kernel could use. For a kernel launched without the
// attribute the wait returns immediately.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

// Early trigger (tensor-core mode product and its staging copy only): the next kernel in the
// stream may be scheduled once every block of this grid has executed it. Its blocks take SMs as
// this grid's blocks exit and run the part before their own pdl_begin(), which reads nothing a
// preceding kernel writes, while the rest of this grid finishes.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// Returns the launch's own status (configuration errors), not errors left pending by earlier work.
template <typename... P, typename... A>
inline cudaError_t launch_k(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t s, A... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

// Raises a kernel's dynamic shared-memory limit to `bytes` when that is above the 48 KiB default
// and above every value set so far for it (`cache`). Several host threads may launch at once
// (concurrent contexts), so the check and the attribute call are serialised. The cache records
// only a size the attribute call accepted; a refused size (above the device's opt-in maximum)
// leaves it unchanged and returns the error, and the launch that needed it must not be made.
template <typename K>
inline cudaError_t raise_smem_limit(K kernel, std::atomic<int>& cache, int bytes) {
  if (bytes <= 48 * 1024 || bytes <= cache.load()) return cudaSuccess;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (bytes <= cache.load()) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) cache.store(bytes);
  return e;
}

// The same with a thread-block cluster of cluster_x blocks along x (grid.x a multiple of it).
template <typename... P, typename... A>
inline void launch_kc(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                      int cluster_x, A... args) {
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = cluster_x;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = cluster_x > 1 ? 2 : 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

// Banded 1D matrix on the device: D(i, start[i] + w) = val[i * width + w].
// Square matrices whose nonzeros all lie within |i - j| <= half also carry a centred copy:
// D(i, i - half + k) = cval[i * cpitch + k] for k < 2 half + 1 (zero where i - half + k is out of
// range), cpitch = (2 half + 4) & ~3 (16-byte rows), rows padded with zeros to a multiple of 8.
// cval is null when the matrix is not of that form. Rows tlo <= i < thi of the centred copy are
// identical (the Toeplitz interior of a matrix on a uniform knot vector); tlo = thi = 0 if none.
template <typename T>
struct BandD {
  int rows, cols, width;
  const int* start;
  const T* val;
  const T* valT;   // the band transposed: valT[w * rows + i] = val[i * width + w]
  const T* cval;
  int half, cpitch;
  int tlo, thi;
};

// Extents of a 3D tensor, x1 fastest: index = i1 + n1 * (i2 + n2 * i3).
struct Dims {
  int n1, n2, n3;
  __host__ __device__ int64_t size() const { return (int64_t)n1 * n2 * n3; }
  __host__ __device__ int get(int axis) const { return axis == 1 ? n1 : (axis == 2 ? n2 : n3); }
  __host__ __device__ Dims with(int axis, int m) const {
    Dims d = *this;
    if (axis == 1) d.n1 = m; else if (axis == 2) d.n2 = m; else d.n3 = m;
    return d;
  }
};

// ---- banded passes (k_band.cu) -----------------------------------------------------------
// Y = c0 (D0 .axis X0) [+ c1 (D1 .axis X1)] [+ cz Z] [+ Dt_axis g  (difference transpose along
// axis `gaxis` of the b^3 tensor g, see k_band.cu)]. X0/X1 have extents `in`; Y has extents
// in.with(axis, D0.rows). Z (may alias Y) and g may be null.
// Batches: nb items (nb <= 1: one), item k of every tensor of the job (X0, X1, Z, g, Y) at
// offset k * bs elements from its pointer.
template <typename T>
struct PassArgs {
  const T* X0; const T* X1;
  BandD<T> D0, D1;
  T c0, c1;
  const T* Z; T cz;
  const T* g; int gaxis; Dims gdims;
  T* Y;
  Dims in;
  int axis;
  int nterms;
  int nb;
  int64_t bs;
  int block;   // FP64 line kernel: threads per block (<= 0: 256); chosen by the setup tuner
  int c0_one;  // c0 == 1 (set by the launcher: the FP64 kernels test this integer instead of
               // comparing c0 per output, an instruction of the slow FP64 pipe)
  int chain;   // two terms with c0 == c1 == 1 (set by the launcher): the FP64 kernels run one
               // FMA chain over both band rows
  // Horner epilogue (one hyper-power step fused into the pass that produces u = A~ t): instead
  // of writing the result v to Y, hmode 1 sets r = hx - v, acc = hx + r (first step, from
  // r = acc = hx); hmode 2 sets r = r - v, acc = acc + r. hr, hacc, hx have Y's layout.
  int hmode;
  T* hr;
  T* hacc;
  const T* hx;
};

// The Horner epilogue of PassArgs as one store: the same operations as writing Y and then
// hp_first / hp_update (vector kernels), so the two routes give the same bits.
template <typename T>
__device__ __forceinline__ void pass_store(const PassArgs<T>& a, int64_t o, T v) {
  if (a.hmode == 0) {
    a.Y[o] = v;
  } else if (a.hmode == 1) {
    const T xi = a.hx[o];
    const T ri = xi - v;
    a.hr[o] = ri;
    a.hacc[o] = xi + ri;
  } else {
    const T ri = a.hr[o] - v;
    a.hr[o] = ri;
    a.hacc[o] += ri;
  }
}
template <typename T>
void band_pass(const PassArgs<T>& a, cudaStream_t s);
// Several independent passes (up to kMaxPassJobs, e.g. one per velocity component) in one launch.
constexpr int kMaxPassJobs = 8;
template <typename T>
void band_pass_multi(const PassArgs<T>* jobs, int njobs, cudaStream_t s);

// delta = sum_c D .c u_c: exact discrete divergence of the velocity coefficients (App. B.2),
// output b^3. (D beta)_i = beta_i - beta_{i-1} with beta_{-1} = beta_a = 0.
// For these three: nb items, item k of every argument tensor at offset k * bs elements.
template <typename T>
void divergence(const T* u1, const T* u2, const T* u3, int a, int b, T* delta, cudaStream_t s,
                int nb = 1, int64_t bs = 0);
// as divergence, and also e = nu delta + q (the argument of the grad-div / pressure term)
template <typename T>
void divergence_plus(const T* u1, const T* u2, const T* u3, int a, int b, T* delta,
                     const T* q, T nu, T* e, cudaStream_t s, int nb = 1, int64_t bs = 0);

// y_c (+)= D^T .c g for the three components (grad of a b^3 field onto velocity coefficients).
template <typename T>
void div_transpose(const T* g, int a, int b, T* y1, T* y2, T* y3, int accumulate,
                   cudaStream_t s, int nb = 1, int64_t bs = 0);

// Quadrature-based forward operator (Sec. 5.3), pointwise step at the n^3 Gauss points (nq per
// direction, x1 fastest): G holds the nine gradient tensors d_d u_c at G + (3c + d) nq^3, P the
// pressure values. In place: G <- W (nu (d_d u_c + d_c u_d) + [c == d] q) (the weighted 2 nu
// eps(u) of a(u, v) plus the pressure of b(v, q), to be contracted with d_d v_c) and
// P <- W div u, with W = w[i1] w[i2] w[i3] the product Gauss weight.
void quad_stress(double* G, double* P, const double* w, int nq, double nu, cudaStream_t s);

// ---- dense mode products (k_dense.cu) ----------------------------------------------------
// Y[l, i, r] = sum_j Op(i, j) X[l, j, r] along `axis` of X (extents `in`), Op(i, j) =
// trans ? U[j * ld + i] : U[i * ld + j], output extents in.with(axis, m).
// If lam1 != null the result is divided by scale * (lam1[i1] + lam2[i2] + lam3[i3]) at output
// index (i1, i2, i3) (fast-diagonalisation scaling, App. A.4).
template <typename T>
struct ModeArgs {
  const T* X; T* Y;
  const T* U; int ld; int trans; int m;
  Dims in; int axis;
  const T* lam1; const T* lam2; const T* lam3; T scale;
  T post;   // if lam1 == null: the result is multiplied by post
  const T* invd;   // if set (FP64 path): the result is multiplied by invd[output index] instead
  int eo_he;       // FP64 path: U's columns are [he even; n - he odd] eigenvectors (0: generic)
  int block;       // FP64 path: target threads per block (<= 0: 512); chosen by the setup tuner
};
// Both return the status of their launch (cudaSuccess, or the error of the shared-memory limit
// or of the launch itself; nothing is launched when the limit cannot be raised).
template <typename T>
cudaError_t mode_product(const ModeArgs<T>& a, cudaStream_t s);
// Several independent mode products (up to kMaxModeJobs) in one launch.
constexpr int kMaxModeJobs = 4;
template <typename T>
cudaError_t mode_product_multi(const ModeArgs<T>* jobs, int njobs, cudaStream_t s);
// Dynamic shared memory (bytes) of the FP64 mode-product kernel for this one job.
int64_t mode_product_smem(const ModeArgs<double>& m);

// Fused FP64 fast-diagonalisation passes (App. A.4), several tensors per launch. The operators
// are square with parity-split eigenvector columns (eo even modes first, eo >= 1), as for
// mode_product with eo_he > 0; each output is computed in the same operation order as by
// mode_product, so the fused and the per-direction forms give identical bits.
//
// Plane pair: the two products along x1 and x2 of every x1-x2 plane, one block or one cluster of
// blocks per plane (the plane and the intermediate stay in shared memory). fwd = 1: Y = (U2^T (x) U1^T) X per plane;
// fwd = 0: Y = post (U2 (x) U1) X (the x2 product first, then x1).
struct FdPlaneArgs {
  const double* X; double* Y;
  const double* U1; const double* U2;   // ld = in.n1 and in.n2
  Dims in;
  int eo1, eo2;
  double post;
};
// Lines along x3: the forward product with U3^T, the eigenvalue scaling (invd, or
// 1 / (scale (lam1 + lam2 + lam3)), or none), and the backward product with U3 (times post).
struct FdLineArgs {
  const double* X; double* Y;
  const double* U3;                      // ld = in.n3
  Dims in;
  int eo3;
  const double* invd;
  const double *lam1, *lam2, *lam3;
  double scale;
  double post;
};
// Shared memory of one plane block (two plane buffers); 0 if the plane does not fit.
int fd_plane_smem(Dims in);
// Both return false without launching if a job does not qualify (plane too large for shared
// memory, no parity split); the caller then uses mode_product_multi.
// cluster: 1, 2 or 4 blocks per plane (a thread-block cluster sharing the plane's intermediate
// through distributed shared memory).
bool fd_plane_multi(const FdPlaneArgs* jobs, int njobs, int fwd, int block, int cluster,
                    cudaStream_t s);
bool fd_line3_multi(const FdLineArgs* jobs, int njobs, int block, cudaStream_t s);

// delta = D_div u (and e = nu delta + q when q is set) and their band pass along x1 in one launch:
// y0 = D .x1 delta, y1 = D .x1 e on the (b, b, b) pressure grid (FP64 contexts, one item).
template <typename T>
void div_band_x1(const T* u1, const T* u2, const T* u3, int a, int b, const T* q, T nu,
                 const BandD<T>& D, T* y0, T* y1, cudaStream_t s);

// Banded Cholesky solves along one direction of a (b, b, b) tensor: y <- post (L L^T)^-1 x (y may
// be x) with L lower triangular of bandwidth p stored as rows lb[i * (p + 1) + (k - i + p)] for
// k in [i - p, i], and inv_diag[i] = 1 / L[i][i] (pressure mass inverse). nb items, item k of x and
// y at k * bs entries. Returns the launch status.
template <typename T>
cudaError_t chol_solve_axis(const T* x, T* y, int b, int p, int axis, const T* lb,
                            const T* inv_diag, T post, cudaStream_t s, int nb = 1,
                            int64_t bs = 0);

// ---- vector kernels (k_vec.cu) -----------------------------------------------------------
// Deterministic dot product: fixed grid, fixed-order tree reduction. Result written to *out
// (device). `partials` holds kDotBlocks values and, in the word after them, a completion counter
// that must be zero before the first call (each call leaves it zero); kDotScratch doubles.
constexpr int kDotBlocks = 512;
constexpr int kDotScratch = kDotBlocks + 2;
// grid of the multi-vector dot products (fixed, so their reductions are deterministic)
constexpr int kMultiDotBlocks = 152 * 4;   // one resident wave (4 blocks per SM)
template <typename T>
void dot(const T* x, const T* y, int64_t n, T* partials, T* out, cudaStream_t s);
// y = a x + b y with a, b from host
template <typename T>
void axpby(T a, const T* x, T b, T* y, int64_t n, cudaStream_t s);
// r = r - u; acc = acc + r  (one hyper-power Horner step, Eq. 2.1 generalised), on nb rows of
// n entries with pitch bs
template <typename T>
void hp_update(T* r, const T* u, T* acc, int64_t n, cudaStream_t s, int nb = 1, int64_t bs = 0);
// first Horner step from r = acc = x: r = x - u; acc = x + r (the same arithmetic as copying x
// into r and acc and then hp_update), on nb rows of n entries with pitch bs
template <typename T>
void hp_first(const T* x, const T* u, T* r, T* acc, int64_t n, cudaStream_t s, int nb = 1,
              int64_t bs = 0);
void copy_async(void* dst, const void* src, size_t bytes, cudaStream_t s);
// nb rows of row_bytes with the same pitch in source and destination (one 2D copy)
void copy_rows(void* dst, const void* src, size_t row_bytes, int nb, size_t pitch_bytes,
               cudaStream_t s);
// y += sign * (*alpha) * x with alpha in device memory
void axpy_dev(const double* alpha, double sign, const double* x, double* y, int64_t n,
              cudaStream_t s);
// y[k] = <V_k, w> for k < nvec (V_k = V + k * ldv); with with_self also y[nvec] = <w, w> from
// the same pass; deterministic; partials: (nvec + 1) * kMultiDotBlocks
void multi_dot(const double* V, int64_t ldv, int nvec, const double* w, int64_t n,
               double* partials, double* out, cudaStream_t s, bool with_self = false);
// out[k] = <V_k, w>, out[nvec + k] = <V_k, z> for k < nvec and out[2 nvec] = <w, w>, from one
// sweep over the vectors; deterministic; partials: (2 nvec + 1) * kMultiDotBlocks
void multi_dot2(const double* V, int64_t ldv, int nvec, const double* w, const double* z,
                int64_t n, double* partials, double* out, cudaStream_t s);
// w += sign * sum_k h[k] V_k (h in device memory; one FMA chain per element from w, in the
// order of k, with the coefficients sign h[k])
void multi_axpy(const double* V, int64_t ldv, int nvec, const double* h, double sign, double* w,
                int64_t n, cudaStream_t s);
// out = (w + sign * sum_k h[k] V_k) * (1 / *div): the chain of multi_axpy, then the product
// (the same bits as multi_axpy followed by scale_inv_dev); out may be w
void multi_axpy_div(const double* V, int64_t ldv, int nvec, const double* h, double sign,
                    const double* w, const double* div, double* out, int64_t n, cudaStream_t s);
// y = x * (1 / *alpha)
void scale_inv_dev(const double* alpha, const double* x, double* y, int64_t n, cudaStream_t s);
void fill_zero(void* dst, size_t bytes, cudaStream_t s);
// out[m] = <x, l1_m (x) l2_m (x) l3_m> for m < nm (extents e1, e2, e3, x1 fastest; device factors
// packed as f[m][3][ld]); deterministic; partials: nm * kMultiDotBlocks.
void sep_dots(const double* x, const double* f, int ld, int nm, int e1, int e2, int e3,
              double* partials, double* out, cudaStream_t s);
// dst (extents e1, e2, e3, x1 fastest) += cf l2 (x) l3 (x) l1 elementwise, in that order of
// operations (device vectors l1, l2, l3 of lengths e1, e2, e3).
void outer3_acc(const double* l1, const double* l2, const double* l3, double cf, double* dst,
                int e1, int e2, int e3, cudaStream_t s);

// MINRES device state and fused kernels (k_vec.cu)
struct MinresState {
  double gamma, gamma_old, eta, eta0, c, c_old, s, s_old;
  double delta, gg;          // dot products written by the dot kernel
  double a1, a2, a3, xcoef;  // update coefficients of the current iteration
  double ratio;
  double tol;                // stopping tolerance (read by the scalar kernel)
  double* ratios;            // per-iteration ratio history (device, `cap` entries)
  int cap;
  int iter, status, done, pad;
};
void minres_scale_z(double* z, MinresState* st, int64_t n, cudaStream_t s);
void minres_lanczos(const double* Kz, const double* v, double* vold_inout, MinresState* st,
                    int64_t n, cudaStream_t s);
void minres_scalars(MinresState* st, cudaStream_t s);
void minres_update(const double* z, double* w_old_inout, const double* w, double* x,
                   MinresState* st, int64_t n, cudaStream_t s);
void minres_init(MinresState* st, cudaStream_t s);

// ---- the saddle-point operator in pair-of-FP32 arithmetic (k_pair.cu) ----------------------
// A value is carried as the unevaluated sum hi + lo of two floats (float2 {hi, lo}), about 48
// significant bits. Band matrices in the centred form of BandD: row i, entry k in [0, 2 H]
// holds D(i, i - H + k) (zero outside the matrix), `pitch` (even) pairs per row, rows padded with
// zeros to a multiple of 8; every term of one launch has the same half width H (1 <= H <= 6).
struct PairBand {
  const float2* c;
  int rows, pitch;
};
// Y = sum_t D_t .axis X_t [+ D^T_gaxis g] (up to two terms). X_t: FP32 (in_f32; the value is
// exact with lo = 0) or pairs; g: pairs on the b^3 grid gdims; Y: FP64 (out_f64) or pairs. Every
// term has X's extents `in`; Y has in.with(axis, rows). nb items, item k of every tensor at k * bs
// elements from its pointer.
struct PairPass {
  const void* X[2];
  PairBand D[2];
  int nterms, in_f32, out_f64;
  const float2* g; int gaxis; Dims gdims;
  void* Y;
  Dims in; int axis;
  int nb; int64_t bs;
};
constexpr int kMaxPairJobs = 8;
// Several passes (up to kMaxPairJobs) of half width H in one launch.
cudaError_t pair_pass_multi(const PairPass* jobs, int njobs, int H, cudaStream_t s);
// delta = D_div u and e = nu delta + q on the (b, b, b) pressure grid from FP32 u1, u2, u3, q,
// formed in pairs, and their band pass along x1: y0 = D .x1 delta, y1 = D .x1 e (pairs); nb
// items at pitch bs. D: centred, half width H.
cudaError_t pair_div_x1(const float* u1, const float* u2, const float* u3, const float* q, int a,
                        int b, float2 nu, const PairBand& D, int H, float2* y0, float2* y1,
                        int nb, int64_t bs, cudaStream_t s);

// float <-> double conversions for the mixed-precision preconditioner
void to_float(const double* x, float* y, int64_t n, cudaStream_t s);
void to_double(const float* x, double* y, int64_t n, cudaStream_t s);

}  // namespace shp
