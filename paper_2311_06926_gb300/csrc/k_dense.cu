// Dense mode products for fast diagonalisation (App. A.4) on the CUDA cores.
//
// A mode product along one direction is a (batched) matrix product: for directions 2 and 3,
// Y[l, i, r] = sum_j X[l, j, r] Op(i, j) with l running over the contiguous leading extents; for
// direction 1, Y[i, r] = sum_j Op(i, j) X[j, r]. Both are written as C[p, q] = sum_k A[p, k] B[k, q]
// with strided operands and tiled through shared memory (64 x 64 output tile, k-chunks of 16,
// 4 x 4 outputs per thread). The fast-diagonalisation division by the eigenvalue sums is fused
// into the epilogue of the last forward product.
#include "internal.h"
#include "profile.h"

namespace shp {
namespace {

constexpr int BP = 64, BQ = 64, BK = 16, NTH = 256;

template <typename T>
struct GemmArgs {
  const T* A; int64_t a_p, a_k, a_b;
  const T* B; int64_t b_k, b_q, b_b;
  T* C; int64_t c_p, c_q, c_b;
  int P, Q, K;
  // optional fast-diagonalisation epilogue
  const T* lam1; const T* lam2; const T* lam3; T scale; Dims out;
  T post;
};

template <typename T>
__global__ void __launch_bounds__(NTH) k_gemm(GemmArgs<T> g) {
  __shared__ T As[BK][BP + 1];
  __shared__ T Bs[BK][BQ + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int p0 = blockIdx.x * BP, q0 = blockIdx.y * BQ;
  const int64_t bz = blockIdx.z;
  const T* A = g.A + bz * g.a_b;
  const T* B = g.B + bz * g.b_b;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  const bool a_pfast = g.a_p == 1;
  const bool b_kfast = g.b_k == 1;
  for (int k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
    for (int t = 0; t < (BP * BK) / NTH; ++t) {
      const int idx = tid + NTH * t;
      int p, k;
      if (a_pfast) { p = idx % BP; k = idx / BP; } else { k = idx % BK; p = idx / BK; }
      const int gp = p0 + p, gk = k0 + k;
      As[k][p] = (gp < g.P && gk < g.K) ? A[gp * g.a_p + gk * g.a_k] : T(0);
    }
#pragma unroll
    for (int t = 0; t < (BQ * BK) / NTH; ++t) {
      const int idx = tid + NTH * t;
      int q, k;
      if (b_kfast) { k = idx % BK; q = idx / BK; } else { q = idx % BQ; k = idx / BQ; }
      const int gq = q0 + q, gk = k0 + k;
      Bs[k][q] = (gq < g.Q && gk < g.K) ? B[gk * g.b_k + gq * g.b_q] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[k][tx + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[k][ty + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
    }
    __syncthreads();
  }
  T* C = g.C + bz * g.c_b;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int p = p0 + tx + 16 * i, q = q0 + ty + 16 * j;
      if (p < g.P && q < g.Q) {
        const int64_t off = p * g.c_p + q * g.c_q;
        T v = acc[i][j];
        if (g.lam1) {
          const int64_t o = off + bz * g.c_b;
          const int i1 = (int)(o % g.out.n1);
          const int64_t t2 = o / g.out.n1;
          const int i2 = (int)(t2 % g.out.n2);
          const int i3 = (int)(t2 / g.out.n2);
          v = v / (g.scale * (g.lam1[i1] + g.lam2[i2] + g.lam3[i3]));
        } else {
          v = v * g.post;
        }
        C[off] = v;
      }
    }
}

}  // namespace

template <typename T>
void mode_product(const ModeArgs<T>& m, cudaStream_t s) {
  GemmArgs<T> g{};
  const Dims in = m.in;
  const int nin = in.get(m.axis);
  const Dims out = in.with(m.axis, m.m);
  // Op(i, j) strides
  const int64_t op_i = m.trans ? 1 : m.ld, op_j = m.trans ? m.ld : 1;
  if (m.axis == 1) {
    // C[i, r] = sum_j Op(i, j) X[j, r]
    g.A = m.U; g.a_p = op_i; g.a_k = op_j; g.a_b = 0;
    g.B = m.X; g.b_k = 1; g.b_q = nin; g.b_b = 0;
    g.C = m.Y; g.c_p = 1; g.c_q = m.m; g.c_b = 0;
    g.P = m.m; g.Q = in.n2 * in.n3; g.K = nin;
    g.lam1 = m.lam1; g.lam2 = m.lam2; g.lam3 = m.lam3; g.scale = m.scale; g.out = out;
    g.post = m.post;
    dim3 grid((g.P + BP - 1) / BP, (g.Q + BQ - 1) / BQ, 1);
    launch_begin(kClassMode, s);
    k_gemm<T><<<grid, NTH, 0, s>>>(g);
    launch_end(kClassMode, s, 2.0 * g.P * g.Q * g.K,
               ((double)in.size() + (double)out.size()) * sizeof(T));
  } else {
    const int64_t L = m.axis == 2 ? in.n1 : (int64_t)in.n1 * in.n2;
    const int R = m.axis == 2 ? in.n3 : 1;
    // C[l, i] = sum_j X[l, j] Op(i, j), batched over r
    g.A = m.X; g.a_p = 1; g.a_k = L; g.a_b = L * nin;
    g.B = m.U; g.b_k = op_j; g.b_q = op_i; g.b_b = 0;
    g.C = m.Y; g.c_p = 1; g.c_q = L; g.c_b = L * m.m;
    g.P = (int)L; g.Q = m.m; g.K = nin;
    g.lam1 = m.lam1; g.lam2 = m.lam2; g.lam3 = m.lam3; g.scale = m.scale; g.out = out;
    g.post = m.post;
    dim3 grid((g.P + BP - 1) / BP, (g.Q + BQ - 1) / BQ, R);
    launch_begin(kClassMode, s);
    k_gemm<T><<<grid, NTH, 0, s>>>(g);
    launch_end(kClassMode, s, 2.0 * g.P * g.Q * g.K * R,
               ((double)in.size() + (double)out.size()) * sizeof(T));
  }
}

template void mode_product<double>(const ModeArgs<double>&, cudaStream_t);
template void mode_product<float>(const ModeArgs<float>&, cudaStream_t);

}  // namespace shp
