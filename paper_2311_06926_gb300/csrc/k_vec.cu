// Vector kernels of the Krylov iteration: deterministic dot products, fused axpys, and the
// preconditioned MINRES recurrences (Lanczos three-term step, Givens QR scalars, update of the
// direction and the iterate) with all scalars kept in device memory.
#include <cmath>

#include "internal.h"
#include "profile.h"

namespace shp {
namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t total) {
  int64_t b = (total + kThreads - 1) / kThreads;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename T>
__device__ T block_sum(T v, T* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  return sh[0];
}

// Stage 1: block b sums elements b*256+t, b*256+t+G*256, ... in a fixed order.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_dot_partial(const T* __restrict__ x,
                                                          const T* __restrict__ y, int64_t n,
                                                          T* __restrict__ partials) {
  pdl_begin();
  __shared__ T sh[kThreads];
  T s = 0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads)
    s += x[i] * y[i];
  const T tot = block_sum(s, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// The two stages in one launch: every block writes its partial sum, and the last block to finish
// (a completion counter in the word after the kDotBlocks partials) sums the partials in the order
// of k_dot_final and resets the counter. The result has the bits of the two-kernel form.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_dot_single(const T* __restrict__ x,
                                                         const T* __restrict__ y, int64_t n,
                                                         T* partials, T* __restrict__ out) {
  pdl_begin();
  __shared__ T sh[kThreads];
  __shared__ int last;
  T s = 0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads)
    s += x[i] * y[i];
  const T tot = block_sum(s, sh);
  unsigned int* ctr = reinterpret_cast<unsigned int*>(partials + kDotBlocks);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = tot;
    __threadfence();
    last = atomicAdd(ctr, 1u) == gridDim.x - 1 ? 1 : 0;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  T s2 = 0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += kThreads) s2 += __ldcg(partials + i);
  const T t2 = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    *out = t2;
    *ctr = 0u;
  }
}

// dst[i1 + e1 (i2 + e2 i3)] += cf l2[i2] l3[i3] l1[i1]: one rank-one term of a separable load.
__global__ void k_outer3_acc(const double* __restrict__ l1, const double* __restrict__ l2,
                             const double* __restrict__ l3, double cf, double* __restrict__ dst,
                             int e1, int e2, int e3) {
  pdl_begin();
  const int64_t total = (int64_t)e1 * e2 * e3;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i1, i2, i3;
    if (total < ((int64_t)1 << 31)) {   // 32-bit division (64-bit division uses the FP64 pipe)
      const int t32 = (int)t, q = t32 / e1;
      i1 = t32 - q * e1;
      i3 = q / e2;
      i2 = q - i3 * e2;
    } else {
      const int64_t q = t / e1;
      i1 = (int)(t - q * e1);
      i2 = (int)(q % e2);
      i3 = (int)(q / e2);
    }
    const double s23 = __dmul_rn(__dmul_rn(cf, l2[i2]), l3[i3]);
    dst[t] = __dadd_rn(dst[t], __dmul_rn(s23, l1[i1]));
  }
}

// Stage 2: one block sums the partials in a fixed order.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_dot_final(const T* __restrict__ partials, int np,
                                                        T* __restrict__ out) {
  pdl_begin();
  __shared__ T sh[kThreads];
  T s = 0;
  for (int i = threadIdx.x; i < np; i += kThreads) s += partials[i];
  const T tot = block_sum(s, sh);
  if (threadIdx.x == 0) *out = tot;
}

template <typename T>
__global__ void k_axpby(T a, const T* __restrict__ x, T b, T* __restrict__ y, int64_t n) {
  pdl_begin();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

// nb rows of n entries with pitch bs (nb == 1: one contiguous range)
template <typename T>
__global__ void k_hp_update(T* __restrict__ r, const T* __restrict__ u, T* __restrict__ acc,
                            int64_t n, int nb, int64_t bs) {
  pdl_begin();
  const int64_t total = n * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = nb > 1 ? t / n : 0;
    const int64_t i = t + k * (bs - n);
    const T ri = r[i] - u[i];
    r[i] = ri;
    acc[i] += ri;
  }
}

template <typename T>
__global__ void k_hp_first(const T* __restrict__ x, const T* __restrict__ u, T* __restrict__ r,
                           T* __restrict__ acc, int64_t n, int nb, int64_t bs) {
  pdl_begin();
  const int64_t total = n * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = nb > 1 ? t / n : 0;
    const int64_t i = t + k * (bs - n);
    const T xi = x[i];
    const T ri = xi - u[i];
    r[i] = ri;
    acc[i] = xi + ri;
  }
}

__global__ void k_to_float(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
  pdl_begin();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

__global__ void k_to_double(const float* __restrict__ x, double* __restrict__ y, int64_t n) {
  pdl_begin();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

__global__ void k_axpy_dev(const double* __restrict__ alpha, double sign,
                           const double* __restrict__ x, double* __restrict__ y, int64_t n) {
  pdl_begin();
  const double a = sign * (*alpha);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

__global__ void k_scale_inv_dev(const double* __restrict__ alpha, const double* __restrict__ x,
                                double* __restrict__ y, int64_t n) {
  pdl_begin();
  const double a = 1.0 / (*alpha);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

// Partial dot products of w with nvec vectors: block b handles the same slice for every vector.
// y[k] = <V_k, w>, NG <= kDotGroup vectors per sweep over the index range: each element of w is
// loaded once per group, every vector has its own accumulator, and a thread handles two
// elements per step, so 2 (NG + 1) independent loads are in flight per thread. Block b of the
// fixed grid of kMultiDotBlocks sums its elements in a fixed order, reduces each vector's sums in
// a fixed tree (warp shuffles, then the warps in order), and stage 2 sums the block partials in a
// fixed order: the result is deterministic.
constexpr int kDotGroup = 8;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Inner products of x with separable tensors T_m = l1_m (x) l2_m (x) l3_m (extents e1, e2, e3,
// x1 fastest), m = k0 .. k0 + NG - 1, whose factors are packed as f[m][3][ld]: the tensors are
// formed on the fly; per-block partial sums in a fixed order, as in k_multi_dot_partial.
template <int NG>
__global__ void __launch_bounds__(kThreads, 4) k_sep_dot_partial(const double* __restrict__ x,
                                                              const double* __restrict__ f,
                                                              int ld, int k0, int e1, int e2,
                                                              int e3,
                                                              double* __restrict__ partials) {
  pdl_begin();
  __shared__ double sh[NG][kThreads / 32];
  double acc[NG];
#pragma unroll
  for (int g = 0; g < NG; ++g) acc[g] = 0.0;
  const double* f0 = f + (int64_t)k0 * 3 * ld;
  const int64_t n = (int64_t)e1 * e2 * e3;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    int i1, i2, i3;
    if (n < ((int64_t)1 << 31)) {   // 32-bit division (64-bit division uses the FP64 pipe)
      const int i32 = (int)i, q = i32 / e1;
      i1 = i32 - q * e1;
      i3 = q / e2;
      i2 = q - i3 * e2;
    } else {
      const int64_t q = i / e1;
      i1 = (int)(i - q * e1);
      i2 = (int)(q % e2);
      i3 = (int)(q / e2);
    }
    const double xv = x[i];
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const double* fg = f0 + (int64_t)g * 3 * ld;
      acc[g] = fma(xv, __ldg(fg + i1) * __ldg(fg + ld + i2) * __ldg(fg + 2 * ld + i3), acc[g]);
    }
  }
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    const double t = warp_sum(acc[g]);
    if (lane == 0) sh[g][warp] = t;
  }
  __syncthreads();
  if ((int)threadIdx.x < NG) {
    double t = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) t += sh[threadIdx.x][k];
    partials[(int64_t)(k0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
  }
}

// SELF: the block also sums w_i^2 in the same order (one more accumulator), written as partial
// row self_row, so <w, w> comes with the products at no extra read of w.
template <int NG, bool SELF>
__global__ void __launch_bounds__(kThreads, 4) k_multi_dot_partial(const double* __restrict__ V,
                                                                int64_t ldv, int k0,
                                                                const double* __restrict__ w,
                                                                int64_t n,
                                                                double* __restrict__ partials,
                                                                int self_row) {
  pdl_begin();
  constexpr int NA = NG + (SELF ? 1 : 0);
  __shared__ double sh[NA][kThreads / 32];
  double acc[NA];
#pragma unroll
  for (int g = 0; g < NA; ++g) acc[g] = 0.0;
  const double* v0 = V + (int64_t)k0 * ldv;
  const int64_t step = (int64_t)gridDim.x * kThreads;
  int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  for (; i + step < n; i += 2 * step) {
    const double wa = w[i], wb = w[i + step];
    double va[NG], vb[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      va[g] = v0[g * ldv + i];
      vb[g] = v0[g * ldv + i + step];
    }
#pragma unroll
    for (int g = 0; g < NG; ++g) acc[g] = fma(vb[g], wb, fma(va[g], wa, acc[g]));
    if (SELF) acc[NG] = fma(wb, wb, fma(wa, wa, acc[NG]));
  }
  if (i < n) {
    const double wa = w[i];
#pragma unroll
    for (int g = 0; g < NG; ++g) acc[g] = fma(v0[g * ldv + i], wa, acc[g]);
    if (SELF) acc[NG] = fma(wa, wa, acc[NG]);
  }
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
#pragma unroll
  for (int g = 0; g < NA; ++g) {
    const double t = warp_sum(acc[g]);
    if (lane == 0) sh[g][warp] = t;
  }
  __syncthreads();
  if ((int)threadIdx.x < NA) {
    double t = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) t += sh[threadIdx.x][k];
    const int row = (int)threadIdx.x < NG ? k0 + (int)threadIdx.x : self_row;
    partials[(int64_t)row * gridDim.x + blockIdx.x] = t;
  }
}

// Products of NG basis vectors with two vectors in one sweep: <V_k, w> (partial row k) and
// <V_k, z> (row nvec + k), and with SELF also <w, w> (row 2 nvec); per-block sums in the fixed
// order of k_multi_dot_partial.
template <int NG, bool SELF>
__global__ void __launch_bounds__(kThreads, 4) k_multi_dot2_partial(const double* __restrict__ V,
                                                                 int64_t ldv, int k0, int nvec,
                                                                 const double* __restrict__ w,
                                                                 const double* __restrict__ z,
                                                                 int64_t n,
                                                                 double* __restrict__ partials) {
  pdl_begin();
  constexpr int NA = 2 * NG + (SELF ? 1 : 0);
  __shared__ double sh[NA][kThreads / 32];
  double acc[NA];
#pragma unroll
  for (int g = 0; g < NA; ++g) acc[g] = 0.0;
  const double* v0 = V + (int64_t)k0 * ldv;
  const int64_t step = (int64_t)gridDim.x * kThreads;
  int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  for (; i + step < n; i += 2 * step) {
    const double wa = w[i], wb = w[i + step], za = z[i], zb = z[i + step];
    double va[NG], vb[NG];
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      va[g] = v0[g * ldv + i];
      vb[g] = v0[g * ldv + i + step];
    }
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      acc[g] = fma(vb[g], wb, fma(va[g], wa, acc[g]));
      acc[NG + g] = fma(vb[g], zb, fma(va[g], za, acc[NG + g]));
    }
    if (SELF) acc[2 * NG] = fma(wb, wb, fma(wa, wa, acc[2 * NG]));
  }
  if (i < n) {
    const double wa = w[i], za = z[i];
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const double va = v0[g * ldv + i];
      acc[g] = fma(va, wa, acc[g]);
      acc[NG + g] = fma(va, za, acc[NG + g]);
    }
    if (SELF) acc[2 * NG] = fma(wa, wa, acc[2 * NG]);
  }
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
#pragma unroll
  for (int g = 0; g < NA; ++g) {
    const double t = warp_sum(acc[g]);
    if (lane == 0) sh[g][warp] = t;
  }
  __syncthreads();
  if ((int)threadIdx.x < NA) {
    double t = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) t += sh[threadIdx.x][k];
    const int g = threadIdx.x;
    const int row = g < NG ? k0 + g : (g < 2 * NG ? nvec + k0 + (g - NG) : 2 * nvec);
    partials[(int64_t)row * gridDim.x + blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kThreads) k_multi_dot_final(const double* __restrict__ partials,
                                                              int np, double* __restrict__ out) {
  pdl_begin();
  __shared__ double sh[kThreads];
  const double* p = partials + (int64_t)blockIdx.x * np;
  double s = 0;
  for (int i = threadIdx.x; i < np; i += kThreads) s += p[i];
  const double tot = block_sum(s, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = tot;
}

// w += sign * sum_k h[k] V_k: coefficients (times sign) staged in shared memory, one FMA chain
// per element starting from w, two elements per thread and step.
constexpr int kAxpyMaxVec = 512;   // restart <= 400 (checked at setup)

// out = (w + sum_k (sign h[k]) V_k) * (1 / *div), the sum one FMA chain from w in the order of k
// (div may be null: no scaling; out may be w).
__global__ void __launch_bounds__(kThreads) k_multi_axpy(const double* __restrict__ V, int64_t ldv,
                                                         int nvec, const double* __restrict__ h,
                                                         double sign, const double* w,
                                                         double* out, const double* div,
                                                         int64_t n) {
  pdl_begin();
  // sign h_k (an exact sign change) and 1 / div once per block: every FP64 instruction counts on
  // this part's FP64 pipe, so each element costs nvec FMAs (and one multiply when scaled)
  __shared__ double hs[kAxpyMaxVec];
  __shared__ double inv;
  for (int k = threadIdx.x; k < nvec; k += kThreads) hs[k] = sign < 0 ? -h[k] : h[k];
  const bool scaled = div != nullptr;
  if (threadIdx.x == 0) inv = scaled ? 1.0 / (*div) : 1.0;
  __syncthreads();
  const double a = inv;
  // two elements per thread and step: two independent FMA chains
  const int64_t step = (int64_t)gridDim.x * kThreads;
  int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  for (; i + step < n; i += 2 * step) {
    const double* v = V + i;
    double r0 = w[i], r1 = w[i + step];
    for (int k = 0; k < nvec; ++k) {
      const double hk = hs[k];
      r0 = fma(hk, v[k * ldv], r0);
      r1 = fma(hk, v[k * ldv + step], r1);
    }
    out[i] = scaled ? a * r0 : r0;
    out[i + step] = scaled ? a * r1 : r1;
  }
  if (i < n) {
    const double* v = V + i;
    double r0 = w[i];
    for (int k = 0; k < nvec; ++k) r0 = fma(hs[k], v[k * ldv], r0);
    out[i] = scaled ? a * r0 : r0;
  }
}

// ---- MINRES ---------------------------------------------------------------------------------
// status codes mirror the public error codes
constexpr int kStatusNonfinite = -3;
constexpr int kStatusNotSpd = -4;
constexpr int kStatusMaxit = -5;

__global__ void k_minres_init(MinresState* st) {
  pdl_begin();
  const double gg = st->gg;
  st->status = 0;
  st->iter = 0;
  st->done = 0;
  st->pad = 0;
  if (!isfinite(gg)) {
    st->status = kStatusNonfinite;
    st->done = 1;
    return;
  }
  if (gg < 0.0) {
    st->status = kStatusNotSpd;
    st->done = 1;
    return;
  }
  st->gamma = sqrt(gg);
  st->gamma_old = 1.0;
  st->eta = st->gamma;
  st->eta0 = st->gamma;
  st->c = st->c_old = 1.0;
  st->s = st->s_old = 0.0;
  st->ratio = 1.0;
  if (st->gamma == 0.0) {       // zero right-hand side: x = 0 is the solution
    st->ratio = 0.0;
    st->done = 1;
  }
}

__global__ void k_minres_scale_z(double* __restrict__ z, const MinresState* __restrict__ st,
                                 int64_t n) {
  pdl_begin();
  if (st->done) return;
  const double inv = 1.0 / st->gamma;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    z[i] *= inv;
}

// v_new = Kz - (delta / gamma) v - (gamma / gamma_old) v_old, written over v_old.
__global__ void k_minres_lanczos(const double* __restrict__ Kz, const double* __restrict__ v,
                                 double* __restrict__ vold, const MinresState* __restrict__ st,
                                 int64_t n) {
  pdl_begin();
  if (st->done) return;
  const double a = st->delta / st->gamma, b = st->gamma / st->gamma_old;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    vold[i] = Kz[i] - a * v[i] - b * vold[i];
}

// Givens QR of the Lanczos tridiagonal: apply the two previous rotations to the new column
// (gamma, delta, gamma_new), form the new rotation, and update the residual estimate |eta|.
__global__ void k_minres_scalars(MinresState* st) {
  pdl_begin();
  st->pad = 0;                   // "update this iteration" flag read by the update kernel
  if (st->done) return;
  if (st->iter >= st->cap) {     // iteration cap: keep the last iterate
    st->status = kStatusMaxit;
    st->done = 1;
    return;
  }
  const double gg = st->gg, delta = st->delta;
  if (!isfinite(gg) || !isfinite(delta)) {
    st->status = kStatusNonfinite;
    st->done = 1;
    return;
  }
  if (gg < 0.0) {
    st->status = kStatusNotSpd;
    st->done = 1;
    return;
  }
  const double gamma = st->gamma, gamma_new = sqrt(gg);
  const double c = st->c, c_old = st->c_old, s = st->s, s_old = st->s_old;
  const double a0 = c * delta - c_old * s * gamma;
  const double a1 = sqrt(a0 * a0 + gamma_new * gamma_new);
  const double a2 = s * delta + c_old * c * gamma;
  const double a3 = s_old * gamma;
  const double c_new = a0 / a1, s_new = gamma_new / a1;
  st->a1 = a1;
  st->a2 = a2;
  st->a3 = a3;
  st->xcoef = c_new * st->eta;
  st->eta = -s_new * st->eta;
  st->ratio = fabs(st->eta) / st->eta0;
  if (st->ratios && st->iter < st->cap) st->ratios[st->iter] = st->ratio;
  st->c_old = c;
  st->c = c_new;
  st->s_old = s;
  st->s = s_new;
  st->gamma_old = gamma;
  st->gamma = gamma_new;
  st->iter += 1;
  st->pad = 1;
  if (st->ratio <= st->tol) st->done = 1;
}

// w_new = (z - a3 w_old - a2 w) / a1 over w_old; x += (c_new eta) w_new.
__global__ void k_minres_update(const double* __restrict__ z, double* __restrict__ wold,
                                const double* __restrict__ w, double* __restrict__ x,
                                const MinresState* __restrict__ st, int64_t n) {
  pdl_begin();
  if (!st->pad) return;
  const double inv = 1.0 / st->a1, a2 = st->a2, a3 = st->a3, xc = st->xcoef;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double wn = (z[i] - a3 * wold[i] - a2 * w[i]) * inv;
    wold[i] = wn;
    x[i] += xc * wn;
  }
}

}  // namespace

template <typename T>
void dot(const T* x, const T* y, int64_t n, T* partials, T* out, cudaStream_t s) {
  launch_begin(kClassVector, s);
  launch_k(k_dot_single<T>, kDotBlocks, kThreads, 0, s, x, y, n, partials, out);
  launch_end(kClassVector, s, 2.0 * (double)n, 2.0 * (double)n * sizeof(T));
}

template <typename T>
void axpby(T a, const T* x, T b, T* y, int64_t n, cudaStream_t s) {
  launch_begin(kClassVector, s);
  launch_k(k_axpby<T>, grid_for(n), kThreads, 0, s, a, x, b, y, n);
  launch_end(kClassVector, s, 3.0 * (double)n, 3.0 * (double)n * sizeof(T));
}

template <typename T>
void hp_update(T* r, const T* u, T* acc, int64_t n, cudaStream_t s, int nb, int64_t bs) {
  if (nb < 1) nb = 1;
  launch_begin(kClassVector, s);
  launch_k(k_hp_update<T>, grid_for(n * nb), kThreads, 0, s, r, u, acc, n, nb, nb > 1 ? bs : n);
  launch_end(kClassVector, s, 2.0 * (double)n * nb, 5.0 * (double)n * nb * sizeof(T));
}

template <typename T>
void hp_first(const T* x, const T* u, T* r, T* acc, int64_t n, cudaStream_t s, int nb, int64_t bs) {
  if (nb < 1) nb = 1;
  launch_begin(kClassVector, s);
  launch_k(k_hp_first<T>, grid_for(n * nb), kThreads, 0, s, x, u, r, acc, n, nb, nb > 1 ? bs : n);
  launch_end(kClassVector, s, 2.0 * (double)n * nb, 4.0 * (double)n * nb * sizeof(T));
}

void copy_async(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
}

void copy_rows(void* dst, const void* src, size_t row_bytes, int nb, size_t pitch_bytes,
               cudaStream_t s) {
  if (nb <= 1) {
    cudaMemcpyAsync(dst, src, row_bytes, cudaMemcpyDeviceToDevice, s);
    return;
  }
  cudaMemcpy2DAsync(dst, pitch_bytes, src, pitch_bytes, row_bytes, nb, cudaMemcpyDeviceToDevice, s);
}

void fill_zero(void* dst, size_t bytes, cudaStream_t s) { cudaMemsetAsync(dst, 0, bytes, s); }

void to_float(const double* x, float* y, int64_t n, cudaStream_t s) {
  launch_begin(kClassVector, s);
  launch_k(k_to_float, grid_for(n), kThreads, 0, s, x, y, n);
  launch_end(kClassVector, s, 0.0, 12.0 * (double)n);
}
void to_double(const float* x, double* y, int64_t n, cudaStream_t s) {
  launch_begin(kClassVector, s);
  launch_k(k_to_double, grid_for(n), kThreads, 0, s, x, y, n);
  launch_end(kClassVector, s, 0.0, 12.0 * (double)n);
}

void axpy_dev(const double* alpha, double sign, const double* x, double* y, int64_t n,
              cudaStream_t s) {
  launch_begin(kClassVector, s);
  launch_k(k_axpy_dev, grid_for(n), kThreads, 0, s, alpha, sign, x, y, n);
  launch_end(kClassVector, s, 2.0 * (double)n, 24.0 * (double)n);
}
void scale_inv_dev(const double* alpha, const double* x, double* y, int64_t n, cudaStream_t s) {
  launch_begin(kClassVector, s);
  launch_k(k_scale_inv_dev, grid_for(n), kThreads, 0, s, alpha, x, y, n);
  launch_end(kClassVector, s, (double)n, 16.0 * (double)n);
}
void multi_dot(const double* V, int64_t ldv, int nvec, const double* w, int64_t n,
               double* partials, double* out, cudaStream_t s, bool with_self) {
  for (int k0 = 0; k0 < nvec; k0 += kDotGroup) {
    const int ng = nvec - k0 < kDotGroup ? nvec - k0 : kDotGroup;
    const bool self = with_self && k0 == 0;
    launch_begin(kClassVector, s);
    switch (ng) {
#define SHP_MDOT(g)                                                                             \
  case g:                                                                                       \
    if (self)                                                                                   \
      launch_k(k_multi_dot_partial<g, true>, kMultiDotBlocks, kThreads, 0, s, V, ldv, k0, w, n, \
               partials, nvec);                                                                 \
    else                                                                                        \
      launch_k(k_multi_dot_partial<g, false>, kMultiDotBlocks, kThreads, 0, s, V, ldv, k0, w,   \
               n, partials, nvec);                                                              \
    break;
      SHP_MDOT(1) SHP_MDOT(2) SHP_MDOT(3) SHP_MDOT(4) SHP_MDOT(5) SHP_MDOT(6) SHP_MDOT(7)
      SHP_MDOT(8)
#undef SHP_MDOT
      default: break;
    }
    launch_end(kClassVector, s, 2.0 * (double)n * (ng + (self ? 1 : 0)),
               8.0 * (double)n * (ng + 1));
  }
  launch_begin(kClassVector, s);
  launch_k(k_multi_dot_final, nvec + (with_self ? 1 : 0), kThreads, 0, s, partials,
           kMultiDotBlocks, out);
  launch_end(kClassVector, s, 0.0, 0.0);
}
void multi_dot2(const double* V, int64_t ldv, int nvec, const double* w, const double* z,
                int64_t n, double* partials, double* out, cudaStream_t s) {
  for (int k0 = 0; k0 < nvec; k0 += kDotGroup) {
    const int ng = nvec - k0 < kDotGroup ? nvec - k0 : kDotGroup;
    const bool self = k0 == 0;
    launch_begin(kClassVector, s);
    switch (ng) {
#define SHP_MDOT2(g)                                                                            \
  case g:                                                                                       \
    if (self)                                                                                   \
      launch_k(k_multi_dot2_partial<g, true>, kMultiDotBlocks, kThreads, 0, s, V, ldv, k0,      \
               nvec, w, z, n, partials);                                                        \
    else                                                                                        \
      launch_k(k_multi_dot2_partial<g, false>, kMultiDotBlocks, kThreads, 0, s, V, ldv, k0,     \
               nvec, w, z, n, partials);                                                        \
    break;
      SHP_MDOT2(1) SHP_MDOT2(2) SHP_MDOT2(3) SHP_MDOT2(4) SHP_MDOT2(5) SHP_MDOT2(6)
      SHP_MDOT2(7) SHP_MDOT2(8)
#undef SHP_MDOT2
      default: break;
    }
    launch_end(kClassVector, s, 4.0 * (double)n * ng + (self ? 2.0 * n : 0.0),
               8.0 * (double)n * (ng + 2));
  }
  launch_begin(kClassVector, s);
  launch_k(k_multi_dot_final, 2 * nvec + 1, kThreads, 0, s, partials, kMultiDotBlocks, out);
  launch_end(kClassVector, s, 0.0, 0.0);
}

void sep_dots(const double* x, const double* f, int ld, int nm, int e1, int e2, int e3,
              double* partials, double* out, cudaStream_t s) {
  const double n = (double)e1 * e2 * e3;
  for (int k0 = 0; k0 < nm; k0 += kDotGroup) {
    const int ng = nm - k0 < kDotGroup ? nm - k0 : kDotGroup;
    launch_begin(kClassVector, s);
    switch (ng) {
#define SHP_SDOT(g)                                                                         \
  case g:                                                                                   \
    launch_k(k_sep_dot_partial<g>, kMultiDotBlocks, kThreads, 0, s, x, f, ld, k0, e1, e2, e3, \
             partials);                                                                     \
    break;
      SHP_SDOT(1) SHP_SDOT(2) SHP_SDOT(3) SHP_SDOT(4) SHP_SDOT(5) SHP_SDOT(6) SHP_SDOT(7)
      SHP_SDOT(8)
#undef SHP_SDOT
      default: break;
    }
    launch_end(kClassVector, s, 4.0 * n * ng, 8.0 * n);
  }
  launch_begin(kClassVector, s);
  launch_k(k_multi_dot_final, nm, kThreads, 0, s, partials, kMultiDotBlocks, out);
  launch_end(kClassVector, s, 0.0, 0.0);
}

void multi_axpy(const double* V, int64_t ldv, int nvec, const double* h, double sign, double* w,
                int64_t n, cudaStream_t s) {
  launch_begin(kClassVector, s);
  launch_k(k_multi_axpy, grid_for(n), kThreads, 0, s, V, ldv, nvec, h, sign,
           static_cast<const double*>(w), w, static_cast<const double*>(nullptr), n);
  launch_end(kClassVector, s, 2.0 * nvec * (double)n, 8.0 * (double)n * (nvec + 2));
}
void multi_axpy_div(const double* V, int64_t ldv, int nvec, const double* h, double sign,
                    const double* w, const double* div, double* out, int64_t n, cudaStream_t s) {
  launch_begin(kClassVector, s);
  launch_k(k_multi_axpy, grid_for(n), kThreads, 0, s, V, ldv, nvec, h, sign, w, out, div, n);
  launch_end(kClassVector, s, 2.0 * nvec * (double)n, 8.0 * (double)n * (nvec + 2));
}

void outer3_acc(const double* l1, const double* l2, const double* l3, double cf, double* dst,
                int e1, int e2, int e3, cudaStream_t s) {
  const int64_t total = (int64_t)e1 * e2 * e3;
  launch_begin(kClassVector, s);
  launch_k(k_outer3_acc, grid_for(total), kThreads, 0, s, l1, l2, l3, cf, dst, e1, e2, e3);
  launch_end(kClassVector, s, 4.0 * (double)total, 16.0 * (double)total);
}

void minres_init(MinresState* st, cudaStream_t s) { launch_begin(kClassVector, s);
  launch_k(k_minres_init, 1, 1, 0, s, st);
  launch_end(kClassVector, s, 0.0, 0.0); }
void minres_scale_z(double* z, MinresState* st, int64_t n, cudaStream_t s) {
  launch_begin(kClassVector, s);
  launch_k(k_minres_scale_z, grid_for(n), kThreads, 0, s, z, st, n);
  launch_end(kClassVector, s, (double)n, 16.0 * (double)n);
}
void minres_lanczos(const double* Kz, const double* v, double* vold, MinresState* st, int64_t n,
                    cudaStream_t s) {
  launch_begin(kClassVector, s);
  launch_k(k_minres_lanczos, grid_for(n), kThreads, 0, s, Kz, v, vold, st, n);
  launch_end(kClassVector, s, 4.0 * (double)n, 32.0 * (double)n);
}
void minres_scalars(MinresState* st, cudaStream_t s) {
  launch_begin(kClassVector, s);
  launch_k(k_minres_scalars, 1, 1, 0, s, st);
  launch_end(kClassVector, s, 0.0, 0.0);
}
void minres_update(const double* z, double* wold, const double* w, double* x, MinresState* st,
                   int64_t n, cudaStream_t s) {
  launch_begin(kClassVector, s);
  launch_k(k_minres_update, grid_for(n), kThreads, 0, s, z, wold, w, x, st, n);
  launch_end(kClassVector, s, 6.0 * (double)n, 48.0 * (double)n);
}

template void dot<double>(const double*, const double*, int64_t, double*, double*, cudaStream_t);
template void dot<float>(const float*, const float*, int64_t, float*, float*, cudaStream_t);
template void axpby<double>(double, const double*, double, double*, int64_t, cudaStream_t);
template void axpby<float>(float, const float*, float, float*, int64_t, cudaStream_t);
template void hp_update<double>(double*, const double*, double*, int64_t, cudaStream_t, int, int64_t);
template void hp_update<float>(float*, const float*, float*, int64_t, cudaStream_t, int, int64_t);
template void hp_first<double>(const double*, const double*, double*, double*, int64_t,
                               cudaStream_t, int, int64_t);
template void hp_first<float>(const float*, const float*, float*, float*, int64_t, cudaStream_t,
                              int, int64_t);

}  // namespace shp
