// Dense mode products for fast diagonalisation (App. A.4) on the CUDA cores.
//
// A mode product along one direction is a (batched) matrix product: for directions 2 and 3,
// Y[l, i, r] = sum_j X[l, j, r] Op(i, j) with l running over the contiguous leading extents; for
// direction 1, Y[i, r] = sum_j Op(i, j) X[j, r]. Both are written as C[p, q] = sum_k A[p, k] B[k, q]
// with strided operands, tiled through shared memory. Several independent products (one per
// velocity component) share one launch: the flat block index selects the product, its batch
// entry and its output tile. The fast-diagonalisation division by the eigenvalue sums is fused
// into the epilogue of the last forward product.
//
// FP32 (CUDA-core fallback of the reduced-precision preconditioner): 64 x 64 tiles, 256 threads,
// 4 x 4 outputs per thread. FP64 uses the row-streaming kernel further below.
#include <algorithm>
#include <atomic>

#include <cooperative_groups.h>

#include "internal.h"
#include "profile.h"

namespace shp {
namespace {

template <typename T>
struct Tile;
template <>
struct Tile<float> {
  static constexpr int BP = 64, BQ = 64, BK = 16, TX = 16, TY = 16, MP = 4, MQ = 4, NTH = 256;
};

template <typename T>
struct GemmArgs {
  const T* A; int64_t a_p, a_k, a_b;
  const T* B; int64_t b_k, b_q, b_b;
  T* C; int64_t c_p, c_q, c_b;
  int P, Q, K, R;
  int tiles_p, tiles_q;
  // optional fast-diagonalisation epilogue
  const T* lam1; const T* lam2; const T* lam3; T scale; Dims out;
  T post;
};

template <typename T>
struct GemmBatch {
  GemmArgs<T> job[kMaxModeJobs];
  int first_block[kMaxModeJobs + 1];
  int njobs;
};

template <typename T>
__global__ void __launch_bounds__(Tile<T>::NTH) k_gemm(const __grid_constant__ GemmBatch<T> gb) {
  pdl_begin();
  using TL = Tile<T>;
  constexpr int BP = TL::BP, BQ = TL::BQ, BK = TL::BK, NTH = TL::NTH;
  __shared__ T As[BK][BP + 1];
  __shared__ T Bs[BK][BQ + 1];
  int jb = 0;
  while (jb + 1 < gb.njobs && (int)blockIdx.x >= gb.first_block[jb + 1]) ++jb;
  const GemmArgs<T>& g = gb.job[jb];
  int local = blockIdx.x - gb.first_block[jb];
  const int tiles = g.tiles_p * g.tiles_q;
  const int bz = local / tiles;
  local -= bz * tiles;
  const int tq = local / g.tiles_p, tp = local - tq * g.tiles_p;
  const int tid = threadIdx.x;
  const int tx = tid % TL::TX, ty = tid / TL::TX;
  const int p0 = tp * BP, q0 = tq * BQ;
  const T* A = g.A + (int64_t)bz * g.a_b;
  const T* B = g.B + (int64_t)bz * g.b_b;
  T acc[TL::MP][TL::MQ];
#pragma unroll
  for (int i = 0; i < TL::MP; ++i)
#pragma unroll
    for (int j = 0; j < TL::MQ; ++j) acc[i][j] = 0;
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
      T av[TL::MP], bv[TL::MQ];
#pragma unroll
      for (int i = 0; i < TL::MP; ++i) av[i] = As[k][tx + TL::TX * i];
#pragma unroll
      for (int j = 0; j < TL::MQ; ++j) bv[j] = Bs[k][ty + TL::TY * j];
#pragma unroll
      for (int i = 0; i < TL::MP; ++i)
#pragma unroll
        for (int j = 0; j < TL::MQ; ++j) acc[i][j] += av[i] * bv[j];
    }
    __syncthreads();
  }
  T* C = g.C + (int64_t)bz * g.c_b;
#pragma unroll
  for (int i = 0; i < TL::MP; ++i)
#pragma unroll
    for (int j = 0; j < TL::MQ; ++j) {
      const int p = p0 + tx + TL::TX * i, q = q0 + ty + TL::TY * j;
      if (p < g.P && q < g.Q) {
        const int64_t off = p * g.c_p + q * g.c_q;
        T v = acc[i][j];
        if (g.lam1) {
          const int64_t o = off + (int64_t)bz * g.c_b;
          int i1, i2, i3;
          if (g.out.size() < ((int64_t)1 << 31)) {   // 32-bit division (64-bit: FP64 pipe)
            const int o32 = (int)o, t2 = o32 / g.out.n1;
            i1 = o32 - t2 * g.out.n1;
            i3 = t2 / g.out.n2;
            i2 = t2 - i3 * g.out.n2;
          } else {
            i1 = (int)(o % g.out.n1);
            const int64_t t2 = o / g.out.n1;
            i2 = (int)(t2 % g.out.n2);
            i3 = (int)(t2 / g.out.n2);
          }
          v = v / (g.scale * (g.lam1[i1] + g.lam2[i2] + g.lam3[i3]));
        } else {
          v = v * g.post;
        }
        C[off] = v;
      }
    }
}

template <typename T>
GemmArgs<T> make_gemm(const ModeArgs<T>& m) {
  using TL = Tile<T>;
  GemmArgs<T> g{};
  const Dims in = m.in;
  const int nin = in.get(m.axis);
  const Dims out = in.with(m.axis, m.m);
  const int64_t op_i = m.trans ? 1 : m.ld, op_j = m.trans ? m.ld : 1;
  if (m.axis == 1) {
    // C[i, r] = sum_j Op(i, j) X[j, r]
    g.A = m.U; g.a_p = op_i; g.a_k = op_j; g.a_b = 0;
    g.B = m.X; g.b_k = 1; g.b_q = nin; g.b_b = 0;
    g.C = m.Y; g.c_p = 1; g.c_q = m.m; g.c_b = 0;
    g.P = m.m; g.Q = in.n2 * in.n3; g.K = nin; g.R = 1;
  } else {
    const int64_t L = m.axis == 2 ? in.n1 : (int64_t)in.n1 * in.n2;
    // C[l, i] = sum_j X[l, j] Op(i, j), batched over r
    g.A = m.X; g.a_p = 1; g.a_k = L; g.a_b = L * nin;
    g.B = m.U; g.b_k = op_j; g.b_q = op_i; g.b_b = 0;
    g.C = m.Y; g.c_p = 1; g.c_q = L; g.c_b = L * m.m;
    g.P = (int)L; g.Q = m.m; g.K = nin; g.R = m.axis == 2 ? in.n3 : 1;
  }
  g.tiles_p = (g.P + TL::BP - 1) / TL::BP;
  g.tiles_q = (g.Q + TL::BQ - 1) / TL::BQ;
  g.lam1 = m.lam1; g.lam2 = m.lam2; g.lam3 = m.lam3; g.scale = m.scale; g.out = out;
  g.post = m.post;
  return g;
}

// ---- FP64 mode products ------------------------------------------------------------------------
// GB300 executes about two FP64 FMA per clock per SM, so an FP64 mode product is bound by the
// FP64 pipe on every mesh size. Extents are used exactly: no padded tiles.
struct RowJob {
  const double* X; double* Y; const double* U;
  int64_t op_i, op_j;      // Op(i, j) = U[i * op_i + j * op_j]
  int64_t L;               // product of the extents before the contracted direction
  int K, m, groups;        // contracted extent, output extent, lines per block
  int64_t R;               // product of the extents after it
  const double* invd;      // optional multiplier per output entry
  const double *lam1, *lam2, *lam3;   // otherwise optional eigenvalue-sum divisor
  double scale;
  Dims out;
  double post;
  int eo;     // > 0: number of even modes (even/odd eigenvector split); 0: generic
  int fwd;    // 1: Op(i, j) = U[j][i] (forward, to mode space); 0: Op(i, j) = U[i][j]
};

struct RowBatch {
  RowJob job[kMaxModeJobs];
  int64_t first[kMaxModeJobs + 1];   // first block of each job
  int njobs;
};

// Shared-memory staged FP64 variant. GB300's FP64 pipe reaches its rate only with many resident
// warps, so every thread computes exactly one output (line, i): a block owns lb neighbouring lines
// of one job and all m outputs of each (lb * m threads, lb about 512 / m). The lines' inputs
// (K x lb) are loaded once, coalesced, into shared memory; Op(i, j) is read through the
// read-only cache. Outputs of products along contiguous lines (L = 1) are staged in shared memory
// for coalesced stores.
// IT: index type of the line and entry arithmetic (int when every job's tensors have fewer than
// 2^31 entries: 64-bit integer division issues FP64-pipe instructions on this part, the pipe the
// kernel is bound by).
template <typename IT>
__global__ void __launch_bounds__(512) k_mode_tile(const __grid_constant__ RowBatch rb) {
  pdl_begin();
  extern __shared__ double shd[];
  int jb = 0;
  while (jb + 1 < rb.njobs && (int64_t)blockIdx.x >= rb.first[jb + 1]) ++jb;
  const RowJob& J = rb.job[jb];
  const int K = J.K, m = J.m;
  const int lb = J.groups;                       // lines per block for this job
  const IT JL = (IT)J.L;
  const IT lines = JL * (IT)J.R;
  const IT line0 = (IT)((int64_t)blockIdx.x - rb.first[jb]) * lb;
  const int nl = (int)(lines - line0 < lb ? lines - line0 : lb);
  const int P = lb + 1;
  double* xs = shd;                 // [K][P]
  double* ys = shd + K * P;         // [m][P] (L == 1 only)
  const int tid = threadIdx.x;
  const int nth = blockDim.x;
  if (JL == 1) {
    for (int idx = tid; idx < K * lb; idx += nth) {
      const int l = idx / K, j = idx - l * K;
      xs[j * P + l] = l < nl ? J.X[(IT)K * (line0 + l) + j] : 0.0;
    }
  } else {
    for (int idx = tid; idx < K * lb; idx += nth) {
      const int l = idx % lb, j = idx / lb;
      double v = 0.0;
      if (l < nl) {
        const IT line = line0 + l;
        const IT r = line / JL, ll = line - r * JL;
        v = J.X[ll + JL * (j + (IT)K * r)];
      }
      xs[j * P + l] = v;
    }
  }
  __syncthreads();
  auto out_index = [&](int l, int i) -> IT {
    if (JL == 1) return (IT)m * (line0 + l) + i;
    const IT line = line0 + l;
    const IT r = line / JL, ll = line - r * JL;
    return ll + JL * ((IT)i + (IT)m * r);
  };
  auto emit = [&](int l, int i, double v) {
    const IT o = out_index(l, i);
    if (J.invd) {
      v *= J.invd[o];
    } else if (J.lam1) {
      const IT t2 = o / J.out.n1, t3 = t2 / J.out.n2;
      const int i1 = (int)(o - t2 * J.out.n1), i2 = (int)(t2 - t3 * J.out.n2);
      v /= J.scale * (J.lam1[i1] + J.lam2[i2] + J.lam3[(int)t3]);
    } else {
      v *= J.post;
    }
    if (JL == 1) ys[i * P + l] = v;
    else J.Y[o] = v;
  };
  if (J.eo == 0) {
    // generic: thread -> (line l, output i), consecutive threads take consecutive i of one line
    for (int q = tid; q < lb * m; q += nth) {
      const int l = q / m, i = q - l * m;
      if (l >= nl) continue;
      double acc = 0.0;
      const double* xcol = xs + l;
      const double* op = J.U + i * J.op_i;
      for (int j = 0; j < K; ++j) acc = fma(__ldg(op + j * J.op_j), xcol[j * P], acc);
      emit(l, i, acc);
    }
  } else if (J.fwd) {
    // even/odd forward: fold each line once (x_k + x_{K-1-k} | x_k - x_{K-1-k}), then every mode
    // is a half-length dot with the top rows of U
    const int he = J.eo, h = K - he;
    double* xf = ys + (J.L == 1 ? m * P : 0);     // [K][P]
    for (int idx = tid; idx < he * lb; idx += nth) {
      const int l = idx % lb, k = idx / lb;
      if (k < h) {
        const double a = xs[k * P + l], b = xs[(K - 1 - k) * P + l];
        xf[k * P + l] = a + b;
        xf[(he + k) * P + l] = a - b;
      } else {
        xf[k * P + l] = xs[k * P + l];           // middle entry of an odd-length line
      }
    }
    __syncthreads();
    for (int q = tid; q < lb * m; q += nth) {
      const int l = q / m, i = q - l * m;
      if (l >= nl) continue;
      const int len = i < he ? he : h;
      const double* xcol = xf + (i < he ? 0 : he * P) + l;
      const double* op = J.U + i;                 // U[k][i], k < len
      double acc = 0.0;
      for (int k = 0; k < len; ++k) acc = fma(__ldg(op + (int64_t)k * J.op_j), xcol[k * P], acc);
      emit(l, i, acc);
    }
  } else {
    // even/odd backward: thread -> (line l, mirrored pair k); a_e over the even modes, a_o over
    // the odd ones; outputs k = a_e + a_o and K-1-k = a_e - a_o
    const int he = J.eo, h = K - he;
    for (int q = tid; q < lb * he; q += nth) {
      const int l = q / he, k = q - l * he;
      if (l >= nl) continue;
      const double* xcol = xs + l;
      const double* row = J.U + (int64_t)k * J.op_i;   // U[k][j]
      double ae = 0.0, ao = 0.0;
      for (int j = 0; j < he; ++j) ae = fma(__ldg(row + j), xcol[j * P], ae);
      if (k < h) {
        for (int j = 0; j < h; ++j) ao = fma(__ldg(row + he + j), xcol[(he + j) * P], ao);
        emit(l, k, ae + ao);
        emit(l, K - 1 - k, ae - ao);
      } else {
        emit(l, k, ae);
      }
    }
  }
  if (JL == 1) {
    __syncthreads();
    for (int idx = tid; idx < m * nl; idx += nth) {
      const int lo = idx / m, io = idx - lo * m;
      J.Y[(IT)m * (line0 + lo) + io] = ys[io * P + lo];
    }
  }
}


// ---- FP64: fused fast-diagonalisation passes ---------------------------------------------------
// At small meshes a single mode-product pass is one partial wave whose load, compute and store
// phases run one after the other, so its fixed latency is comparable to its FP64 work. The fused
// kernels keep the intermediate of two (or three) consecutive passes in shared memory: the x1 and
// x2 products of one x1-x2 plane (one block per plane), and the forward x3 product, the
// eigenvalue scaling and the backward x3 product of a group of x3 lines. Every output is
// computed with the operations and the order of k_mode_tile (even/odd fold, half-length dots
// from k = 0 upward, mirrored pairs a_e +- a_o), so the results are bit-identical.
struct PlaneJob {
  const double* X; double* Y;
  const double* U1; const double* U2;
  int n1, n2;
  int eo1, eo2;
  double post;
};

struct PlaneBatch {
  PlaneJob job[kMaxModeJobs];
  int first[kMaxModeJobs + 1];   // first block (plane) of each job
  int njobs;
  int fwd;
};

// Store v at the same shared-memory offset as p in block `rank` of this cluster.
__device__ __forceinline__ void st_peer(const double* p, int rank, double v) {
  const uint32_t local = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t remote;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(rank));
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(remote), "d"(v) : "memory");
}

// One cluster of cs blocks per plane (cs = 1, 2, 4). Forward: block r loads and folds the x1
// rows of its slice, computes their x1 products and stores them into the plane buffer of every
// block of the cluster; after the cluster barrier each block folds the whole intermediate along x2
// and computes its slice of the x2 outputs. Backward: block r takes a slice of the x1 columns for
// the x2 products (stored to every block), then a slice of the rows for the x1 products.
__global__ void __launch_bounds__(512) k_fd_plane(const __grid_constant__ PlaneBatch pb) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int cs = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  pdl_begin();
  extern __shared__ double shd[];
  const int pidx = (int)blockIdx.x / cs;
  int jb = 0;
  while (jb + 1 < pb.njobs && pidx >= pb.first[jb + 1]) ++jb;
  const PlaneJob& J = pb.job[jb];
  const int plane = pidx - pb.first[jb];
  const int n1 = J.n1, n2 = J.n2, np = n1 * n2;
  double* B0 = shd;        // [n2][n1], x1 fastest
  double* B1 = shd + np;
  const int tid = threadIdx.x, nth = blockDim.x;
  const double* X = J.X + (int64_t)plane * np;
  double* Y = J.Y + (int64_t)plane * np;
  const int he1 = J.eo1, h1 = n1 - he1, he2 = J.eo2, h2 = n2 - he2;
  const int r0 = n2 * rank / cs, r1 = n2 * (rank + 1) / cs;   // this block's x1 rows
  if (cs > 1) cl.sync();   // every block of the cluster runs before any store into it
  if (pb.fwd) {
    const int nr = r1 - r0;
    for (int idx = tid; idx < nr * n1; idx += nth) B0[r0 * n1 + idx] = X[r0 * n1 + idx];
    __syncthreads();
    // fold the x1 rows: (x_k + x_{n1-1-k} | x_k - x_{n1-1-k}), middle entry kept
    for (int idx = tid; idx < he1 * nr; idx += nth) {
      const int j2 = r0 + idx / he1, k = idx - (idx / he1) * he1;
      const double* row = B0 + j2 * n1;
      double* f = B1 + j2 * n1;
      if (k < h1) {
        const double a = row[k], b = row[n1 - 1 - k];
        f[k] = a + b;
        f[he1 + k] = a - b;
      } else {
        f[k] = row[k];
      }
    }
    __syncthreads();
    // x1 products of the rows: T[j2][i1] = sum_k U1[k][i1] f_{j2}[k], into every block's B0
    for (int q = tid; q < nr * n1; q += nth) {
      const int j2 = r0 + q / n1, i1 = q - (q / n1) * n1;
      const int len = i1 < he1 ? he1 : h1;
      const double* xr = B1 + j2 * n1 + (i1 < he1 ? 0 : he1);
      const double* op = J.U1 + i1;
      double acc = 0.0;
      for (int k = 0; k < len; ++k) acc = fma(__ldg(op + k * n1), xr[k], acc);
      B0[j2 * n1 + i1] = acc;
      for (int t = 1, r = rank + 1; t < cs; ++t, ++r)
        st_peer(B0 + j2 * n1 + i1, r < cs ? r : r - cs, acc);
    }
    if (cs > 1) cl.sync(); else __syncthreads();
    // fold every x2 column of the intermediate
    for (int idx = tid; idx < he2 * n1; idx += nth) {
      const int k = idx / n1, i1 = idx - k * n1;
      if (k < h2) {
        const double a = B0[k * n1 + i1], b = B0[(n2 - 1 - k) * n1 + i1];
        B1[k * n1 + i1] = a + b;
        B1[(he2 + k) * n1 + i1] = a - b;
      } else {
        B1[k * n1 + i1] = B0[k * n1 + i1];
      }
    }
    __syncthreads();
    // this block's x2 outputs i2 in [r0, r1), stored coalesced (i1 fastest)
    for (int q = tid; q < nr * n1; q += nth) {
      const int i2 = r0 + q / n1, i1 = q - (q / n1) * n1;
      const int len = i2 < he2 ? he2 : h2;
      const double* xc = B1 + (i2 < he2 ? 0 : he2) * n1 + i1;
      const double* op = J.U2 + i2;
      double acc = 0.0;
      for (int k = 0; k < len; ++k) acc = fma(__ldg(op + k * n2), xc[k * n1], acc);
      Y[i2 * n1 + i1] = acc * J.post;
    }
  } else {
    const int c0 = n1 * rank / cs, c1 = n1 * (rank + 1) / cs, nc = c1 - c0;   // x1 columns
    for (int idx = tid; idx < n2 * nc; idx += nth) {
      const int j2 = idx / nc, i1 = c0 + (idx - (idx / nc) * nc);
      B0[j2 * n1 + i1] = X[j2 * n1 + i1];
    }
    __syncthreads();
    // backward x2: column i1, mirrored output pair (k, n2-1-k) from a_e (even modes) and a_o,
    // into every block's B1
    for (int q = tid; q < he2 * nc; q += nth) {
      const int k = q / nc, i1 = c0 + (q - (q / nc) * nc);
      const double* xc = B0 + i1;
      const double* row = J.U2 + k * n2;
      double ae = 0.0, ao = 0.0;
      for (int j = 0; j < he2; ++j) ae = fma(__ldg(row + j), xc[j * n1], ae);
      if (k < h2) {
        for (int j = 0; j < h2; ++j) ao = fma(__ldg(row + he2 + j), xc[(he2 + j) * n1], ao);
        const double vp = ae + ao, vm = ae - ao;
        B1[k * n1 + i1] = vp;
        B1[(n2 - 1 - k) * n1 + i1] = vm;
        for (int t = 1, r = rank + 1; t < cs; ++t, ++r) {
          const int rr = r < cs ? r : r - cs;
          st_peer(B1 + k * n1 + i1, rr, vp);
          st_peer(B1 + (n2 - 1 - k) * n1 + i1, rr, vm);
        }
      } else {
        B1[k * n1 + i1] = ae;
        for (int t = 1, r = rank + 1; t < cs; ++t, ++r)
          st_peer(B1 + k * n1 + i1, r < cs ? r : r - cs, ae);
      }
    }
    if (cs > 1) cl.sync(); else __syncthreads();
    // backward x1 of this block's rows k2 in [r0, r1): mirrored pair (k, n1-1-k)
    const int nr = r1 - r0;
    for (int q = tid; q < nr * he1; q += nth) {
      const int k2 = r0 + q / he1, k = q - (q / he1) * he1;
      const double* xr = B1 + k2 * n1;
      const double* row = J.U1 + k * n1;
      double ae = 0.0, ao = 0.0;
      for (int j = 0; j < he1; ++j) ae = fma(__ldg(row + j), xr[j], ae);
      double* y = Y + k2 * n1;
      if (k < h1) {
        for (int j = 0; j < h1; ++j) ao = fma(__ldg(row + he1 + j), xr[he1 + j], ao);
        y[k] = (ae + ao) * J.post;
        y[n1 - 1 - k] = (ae - ao) * J.post;
      } else {
        y[k] = ae * J.post;
      }
    }
  }
}

struct LineJob {
  const double* X; double* Y; const double* U;
  int64_t L;             // lines: n1 * n2 (stride of x3)
  int K, eo, lb;         // extent along x3, even modes, lines per block
  int n1;                // to split a line index into (i1, i2)
  const double* invd;
  const double *lam1, *lam2, *lam3;
  double scale;
  double post;
};

struct LineBatch {
  LineJob job[kMaxModeJobs];
  int64_t first[kMaxModeJobs + 1];
  int njobs;
};

__global__ void __launch_bounds__(512) k_fd_line3(const __grid_constant__ LineBatch lbt) {
  pdl_begin();
  extern __shared__ double shd[];
  int jb = 0;
  while (jb + 1 < lbt.njobs && (int64_t)blockIdx.x >= lbt.first[jb + 1]) ++jb;
  const LineJob& J = lbt.job[jb];
  const int K = J.K, nlb = J.lb, P = nlb + 1;
  const int64_t line0 = ((int64_t)blockIdx.x - lbt.first[jb]) * nlb;
  const int nl = (int)(J.L - line0 < nlb ? J.L - line0 : nlb);
  double* xs = shd;             // [K][P] input lines
  double* xf = shd + K * P;     // [K][P] folded
  double* ms = xf + K * P;      // [K][P] scaled mode coefficients
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int idx = tid; idx < K * nlb; idx += nth) {
    const int l = idx % nlb, j = idx / nlb;
    xs[j * P + l] = l < nl ? J.X[line0 + l + J.L * j] : 0.0;
  }
  __syncthreads();
  const int he = J.eo, h = K - he;
  for (int idx = tid; idx < he * nlb; idx += nth) {
    const int l = idx % nlb, k = idx / nlb;
    if (k < h) {
      const double a = xs[k * P + l], b = xs[(K - 1 - k) * P + l];
      xf[k * P + l] = a + b;
      xf[(he + k) * P + l] = a - b;
    } else {
      xf[k * P + l] = xs[k * P + l];
    }
  }
  __syncthreads();
  for (int q = tid; q < nlb * K; q += nth) {
    const int l = q / K, i = q - l * K;
    if (l >= nl) continue;
    const int len = i < he ? he : h;
    const double* xcol = xf + (i < he ? 0 : he * P) + l;
    const double* op = J.U + i;
    double acc = 0.0;
    for (int k = 0; k < len; ++k) acc = fma(__ldg(op + (int64_t)k * K), xcol[k * P], acc);
    double v = acc;
    if (J.invd) {
      v *= J.invd[line0 + l + J.L * i];
    } else if (J.lam1) {
      const int64_t line = line0 + l;
      const int i1 = (int)(line % J.n1), i2 = (int)(line / J.n1);
      v /= J.scale * (J.lam1[i1] + J.lam2[i2] + J.lam3[i]);
    }
    ms[i * P + l] = v;
  }
  __syncthreads();
  for (int q = tid; q < nlb * he; q += nth) {
    const int l = q / he, k = q - l * he;
    if (l >= nl) continue;
    const double* xcol = ms + l;
    const double* row = J.U + (int64_t)k * K;
    double ae = 0.0, ao = 0.0;
    for (int j = 0; j < he; ++j) ae = fma(__ldg(row + j), xcol[j * P], ae);
    double* y = J.Y + line0 + l;
    if (k < h) {
      for (int j = 0; j < h; ++j) ao = fma(__ldg(row + he + j), xcol[(he + j) * P], ao);
      y[J.L * k] = (ae + ao) * J.post;
      y[J.L * (K - 1 - k)] = (ae - ao) * J.post;
    } else {
      y[J.L * k] = ae * J.post;
    }
  }
}
}  // namespace

// Lines per block of k_mode_tile for one job, and the dynamic shared memory that job needs:
// inputs [K][groups + 1]; outputs staged when the lines are contiguous (L == 1); folded inputs
// (even/odd forward).
namespace {
int mode_tile_target(const ModeArgs<double>& m) {
  return m.block > 0 ? std::min(m.block, 512) : 512;
}
int mode_tile_groups(const ModeArgs<double>& m, int target) {
  // threads per line: one per output, or one per mirrored output pair (even/odd backward)
  const int tpl = (m.eo_he && !m.trans) ? m.eo_he : m.m;
  return tpl >= target ? 1 : target / tpl;
}
int64_t mode_tile_smem(const ModeArgs<double>& m, int target) {
  const int K = m.in.get(m.axis);
  const int groups = mode_tile_groups(m, target);
  // contiguous lines (stride 1 between the lines' first elements: axis 1, or axis 2 with n1 = 1)
  const int64_t L = m.axis == 1 ? 1 : (m.axis == 2 ? m.in.n1 : (int64_t)m.in.n1 * m.in.n2);
  return (int64_t)(K + (L == 1 ? m.m : 0) + ((m.eo_he && m.trans) ? K : 0)) * (groups + 1) *
         (int64_t)sizeof(double);
}
}  // namespace

int64_t mode_product_smem(const ModeArgs<double>& m) {
  return mode_tile_smem(m, mode_tile_target(m));
}

template <>
cudaError_t mode_product_multi<double>(const ModeArgs<double>* jobs, int njobs, cudaStream_t s) {
  RowBatch rb{};
  rb.njobs = njobs;
  int blocks = 0, smem = 0, threads = 32;
  // threads per block (target): a block holds target / (threads per line) whole lines
  const int target = jobs[0].block > 0 ? std::min(jobs[0].block, 512) : 512;
  double flops = 0, bytes = 0;
  int first_block[kMaxModeJobs + 1];
  for (int j = 0; j < njobs; ++j) {
    const ModeArgs<double>& m = jobs[j];
    RowJob& J = rb.job[j];
    const Dims in = m.in;
    J.X = m.X;
    J.Y = m.Y;
    J.U = m.U;
    J.op_i = m.trans ? 1 : m.ld;
    J.op_j = m.trans ? m.ld : 1;
    J.K = in.get(m.axis);
    J.m = m.m;
    J.L = m.axis == 1 ? 1 : (m.axis == 2 ? in.n1 : (int64_t)in.n1 * in.n2);
    J.R = m.axis == 1 ? (int64_t)in.n2 * in.n3 : (m.axis == 2 ? in.n3 : 1);
    J.eo = m.eo_he;
    J.fwd = m.trans ? 1 : 0;
    // threads per line: one per output, or one per mirrored output pair (even/odd backward)
    const int tpl = (J.eo && !J.fwd) ? J.eo : m.m;
    J.groups = mode_tile_groups(m, target);  // lines per block
    J.invd = m.invd;
    J.lam1 = m.invd ? nullptr : m.lam1;
    J.lam2 = m.lam2;
    J.lam3 = m.lam3;
    J.scale = m.scale;
    J.out = in.with(m.axis, m.m);
    J.post = m.lam1 ? 1.0 : m.post;
    first_block[j] = blocks;
    blocks += (int)((J.L * J.R + J.groups - 1) / J.groups);
    threads = std::max(threads, std::min(target, ((J.groups * tpl + 31) / 32) * 32));
    const int64_t sm = mode_tile_smem(m, target);
    if (sm > 1024 * 1024) return cudaErrorInvalidValue;
    smem = sm > smem ? (int)sm : smem;
    if (J.eo) {   // even/odd split: two half-size products per line
      const double he = J.eo, ho = J.K - J.eo;
      flops += 2.0 * J.L * J.R * (he * he + ho * ho);
    } else {
      flops += 2.0 * J.L * J.R * (double)J.K * J.m;
    }
    bytes += ((double)in.size() + (double)in.with(m.axis, m.m).size()) * sizeof(double);
  }
  first_block[njobs] = blocks;
  for (int j = 0; j <= njobs; ++j) rb.first[j] = first_block[j];
  // 32-bit entry arithmetic when every tensor of the launch has fewer than 2^31 entries
  bool i32 = true;
  for (int j = 0; j < njobs; ++j) {
    const ModeArgs<double>& m = jobs[j];
    if (std::max(m.in.size(), m.in.with(m.axis, m.m).size()) + 1024 >= ((int64_t)1 << 31))
      i32 = false;
  }
  static std::atomic<int> attr32{0}, attr64{0};
  const cudaError_t e = i32 ? raise_smem_limit(k_mode_tile<int>, attr32, smem)
                            : raise_smem_limit(k_mode_tile<int64_t>, attr64, smem);
  if (e != cudaSuccess) return e;
  launch_begin(kClassMode, s);
  const cudaError_t l = i32 ? launch_k(k_mode_tile<int>, blocks, threads, smem, s, rb)
                            : launch_k(k_mode_tile<int64_t>, blocks, threads, smem, s, rb);
  launch_end(kClassMode, s, flops, bytes);
  return l;
}


int fd_plane_smem(Dims in) {
  const int64_t bytes = 2 * (int64_t)in.n1 * in.n2 * (int64_t)sizeof(double);
  return bytes <= 200 * 1024 ? (int)bytes : 0;
}

namespace {
double eo_flops(int K, int he) {
  const double e = he, o = K - he;
  return 2.0 * (e * e + o * o);
}
std::atomic<int> g_plane_attr{0};
}  // namespace

bool fd_plane_multi(const FdPlaneArgs* jobs, int njobs, int fwd, int block, int cluster,
                    cudaStream_t s) {
  PlaneBatch pb{};
  pb.njobs = njobs;
  pb.fwd = fwd;
  int blocks = 0, smem = 0, work = 32;
  double flops = 0, bytes = 0;
  for (int j = 0; j < njobs; ++j) {
    const FdPlaneArgs& a = jobs[j];
    PlaneJob& J = pb.job[j];
    // outputs (forward) or mirrored pairs (backward) of one block's slice in its larger pass
    const int rows = (a.in.n2 + cluster - 1) / cluster, cols = (a.in.n1 + cluster - 1) / cluster;
    work = std::max(work, fwd ? rows * a.in.n1 : std::max(a.eo2 * cols, rows * a.eo1));
    J.X = a.X;
    J.Y = a.Y;
    J.U1 = a.U1;
    J.U2 = a.U2;
    J.n1 = a.in.n1;
    J.n2 = a.in.n2;
    J.eo1 = a.eo1;
    J.eo2 = a.eo2;
    J.post = a.post;
    pb.first[j] = blocks;
    blocks += a.in.n3;
    const int sm = fd_plane_smem(a.in);
    if (sm == 0 || a.eo1 < 1 || a.eo2 < 1) return false;
    smem = std::max(smem, sm);
    flops += (double)a.in.n3 *
             (a.in.n2 * eo_flops(a.in.n1, a.eo1) + a.in.n1 * eo_flops(a.in.n2, a.eo2));
    bytes += 2.0 * (double)a.in.size() * sizeof(double);
  }
  pb.first[njobs] = blocks;
  if (cluster != 1 && cluster != 2 && cluster != 4) return false;
  // one thread per output of the block's slice (whole warps, at most 512), so every pass is a
  // single round of dot products; with more blocks per plane than the tuned size, block caps it
  const int cap = block > 0 ? std::min(block, 512) : 512;
  const int fit = std::min(512, (work + 31) / 32 * 32);
  const int threads = cluster > 1 ? fit : std::min(cap, fit);
  raise_smem_limit(k_fd_plane, g_plane_attr, smem);
  launch_begin(kClassMode, s);
  launch_kc(k_fd_plane, blocks * cluster, threads, smem, s, cluster, pb);
  launch_end(kClassMode, s, flops, bytes);
  return true;
}

bool fd_line3_multi(const FdLineArgs* jobs, int njobs, int block, cudaStream_t s) {
  LineBatch lbt{};
  lbt.njobs = njobs;
  const int target = block > 0 ? std::min(block, 512) : 512;
  int64_t blocks = 0;
  int smem = 0, threads = 32;
  double flops = 0, bytes = 0;
  for (int j = 0; j < njobs; ++j) {
    const FdLineArgs& a = jobs[j];
    LineJob& J = lbt.job[j];
    J.X = a.X;
    J.Y = a.Y;
    J.U = a.U3;
    J.L = (int64_t)a.in.n1 * a.in.n2;
    J.K = a.in.n3;
    J.eo = a.eo3;
    J.lb = J.K >= target ? 1 : target / J.K;
    J.n1 = a.in.n1;
    J.invd = a.invd;
    J.lam1 = a.invd ? nullptr : a.lam1;
    J.lam2 = a.lam2;
    J.lam3 = a.lam3;
    J.scale = a.scale;
    J.post = a.post;
    if (a.eo3 < 1) return false;
    lbt.first[j] = blocks;
    blocks += (J.L + J.lb - 1) / J.lb;
    smem = std::max(smem, 3 * J.K * (J.lb + 1) * (int)sizeof(double));
    threads = std::max(threads, std::min(target, ((J.lb * J.K + 31) / 32) * 32));
    flops += 2.0 * (double)J.L * eo_flops(J.K, J.eo);
    bytes += 2.0 * (double)a.in.size() * sizeof(double);
  }
  lbt.first[njobs] = blocks;
  static std::atomic<int> attr{0};
  raise_smem_limit(k_fd_line3, attr, smem);
  launch_begin(kClassMode, s);
  launch_k(k_fd_line3, (int)blocks, threads, smem, s, lbt);
  launch_end(kClassMode, s, flops, bytes);
  return true;
}

template <typename T>
cudaError_t mode_product_multi(const ModeArgs<T>* jobs, int njobs, cudaStream_t s) {
  GemmBatch<T> gb{};
  gb.njobs = njobs;
  int blocks = 0;
  double flops = 0, bytes = 0;
  for (int j = 0; j < njobs; ++j) {
    gb.job[j] = make_gemm<T>(jobs[j]);
    gb.first_block[j] = blocks;
    blocks += gb.job[j].tiles_p * gb.job[j].tiles_q * gb.job[j].R;
    const GemmArgs<T>& g = gb.job[j];
    flops += 2.0 * g.P * g.Q * g.K * g.R;
    bytes += ((double)jobs[j].in.size() + (double)jobs[j].in.with(jobs[j].axis, jobs[j].m).size()) *
             sizeof(T);
  }
  gb.first_block[njobs] = blocks;
  launch_begin(kClassMode, s);
  const cudaError_t l = launch_k(k_gemm<T>, blocks, Tile<T>::NTH, 0, s, gb);
  launch_end(kClassMode, s, flops, bytes);
  return l;
}

template <typename T>
cudaError_t mode_product(const ModeArgs<T>& m, cudaStream_t s) {
  return mode_product_multi<T>(&m, 1, s);
}

template cudaError_t mode_product<double>(const ModeArgs<double>&, cudaStream_t);
template cudaError_t mode_product<float>(const ModeArgs<float>&, cudaStream_t);
template cudaError_t mode_product_multi<float>(const ModeArgs<float>*, int, cudaStream_t);

}  // namespace shp
