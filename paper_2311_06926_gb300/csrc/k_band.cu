// Banded Kronecker passes (sum factorisation of App. A.2 with banded 1D factors, Sec. 3.3) and
// the exact discrete divergence / its transpose (App. B.2).
//
// One pass multiplies a 3D tensor along one parametric direction by a banded 1D matrix: each
// output entry is a short dot product of the band row with the input line, read through the
// read-only cache. A pass may sum two such products and add an extra tensor and a difference
// term, so that a whole Kronecker sum is evaluated in few passes.
#include <algorithm>

#include "internal.h"
#include "profile.h"

namespace shp {
namespace {

inline int grid_for(int64_t total, int threads) {
  int64_t b = (total + threads - 1) / threads;
  const int64_t cap = 152 * 32;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename T>
struct PassBatch {
  PassArgs<T> job[kMaxPassJobs];
  int first_block[kMaxPassJobs + 1];
  int njobs;
  int seg;     // outputs per thread along the band direction
  int flat1;   // FP64: passes along x1 enumerate (line, row) with the row fastest
  int w7[kMaxPassJobs];   // FP64, launch width 9: the job's bands have width 7 (passes along x2
                          // or x3), so its chains run over 7 entries instead of 9 zero-padded
};

// Each thread computes a segment of `seg` consecutive outputs along the band direction of one
// line (a fixed position in the other two directions), so consecutive outputs reuse the band
// window of inputs from L1 instead of re-reading it from L2. A warp covers 32 neighbouring lines
// (consecutive x1 for passes along x2 or x3: coalesced), all at the same segment, so the band
// rows it reads are shared (broadcast). The flat block index selects the job. FP32 passes are
// bandwidth bound and use 32 outputs per thread; FP64 passes are bound by the FP64 pipe and use
// one output per thread for the most parallelism.
template <typename T>
constexpr int seg_len() { return sizeof(T) == 4 ? 32 : 1; }

// One FMA chain per band row: the FP64 passes are bound by the FP64 pipe, where every add or
// multiply besides the FMAs costs as much as an FMA (the pipe has the warps to hide the chain's
// latency).
template <int W, typename T, typename IT>
__device__ __forceinline__ T band_dot(const BandD<T>& D, int i, const T* __restrict__ X, IT base,
                                      IT stride, T sum = T(0)) {
  const int s0 = __ldg(D.start + i);
  const T* x = X + (base + (IT)s0 * stride);
  if (W > 0) {
    const T* v = D.val + (int64_t)i * W;
#pragma unroll
    for (int w = 0; w < W; ++w) sum = fma(__ldg(v + w), __ldg(x + (IT)w * stride), sum);
  } else {
    const T* v = D.val + (int64_t)i * D.width;
    for (int w = 0; w < D.width; ++w) sum = fma(__ldg(v + w), __ldg(x + (IT)w * stride), sum);
  }
  return sum;
}

// Passes along x1 with flat1 set: threads enumerate (line, row) with the row fastest, so a warp
// reads a contiguous stretch of the input and writes a contiguous stretch of the output; the band
// coefficients come from the transposed copy of the band (valT, [w][row]) through the read-only
// cache, so that lanes with consecutive rows read consecutive words. (An earlier form staged
// them in shared memory per block: with one output per thread that staging, 2 W m values per
// block, cost more instructions than the FMAs.)
// IT: index type of the thread's (line, row) arithmetic: int when every job's outputs (all items)
// and tensors fit below 2^31, so that no 64-bit division runs (on this part 64-bit integer
// division issues FP64-pipe instructions, the pipe these FP64 passes are bound by); int64_t
// otherwise. Item offsets k * bs are always 64-bit.
template <typename T, int W, typename IT>
__device__ __forceinline__ void band_pass_flat_x1(const PassArgs<T>& a, IT t) {
  const int m = a.D0.rows;
  const Dims out = a.in.with(1, m);
  const int nb = a.nb > 1 ? a.nb : 1;
  const IT per = (IT)out.size();
  if (t >= per * nb) return;
  const IT lines = per / m;
  IT line = t / m;
  const int i = (int)(t - line * m);
  int64_t kb = 0;   // item offset
  if (nb > 1) {
    const IT k = line / lines;
    kb = (int64_t)k * a.bs;
    line -= k * lines;
  }
  const T* c0 = a.D0.valT + i;
  const int64_t base_in = kb + (int64_t)((IT)a.in.n1 * line);
  const T* x0 = a.X0 + base_in + __ldg(a.D0.start + i);
  T acc = 0;
#pragma unroll
  for (int w = 0; w < W; ++w) acc = fma(__ldg(c0 + w * m), __ldg(x0 + w), acc);
  if (a.chain) {
    const T* c1 = a.D1.valT + i;
    const T* x1 = a.X1 + base_in + __ldg(a.D1.start + i);
#pragma unroll
    for (int w = 0; w < W; ++w) acc = fma(__ldg(c1 + w * m), __ldg(x1 + w), acc);
  } else {
    if (!a.c0_one) acc *= a.c0;   // (a product with 1 is exact: skipped)
    if (a.nterms > 1) {
      const T* c1 = a.D1.valT + i;
      const T* x1 = a.X1 + base_in + __ldg(a.D1.start + i);
      T u = 0;
#pragma unroll
      for (int w = 0; w < W; ++w) u = fma(__ldg(c1 + w * m), __ldg(x1 + w), u);
      acc = fma(a.c1, u, acc);
    }
  }
  const int64_t o = kb + (int64_t)((IT)m * line + i);
  if (a.Z) acc += a.cz * a.Z[o];
  if (a.g) {
    // g has extents b^3; along x1 the output's own index is i, the line is (i2, i3)
    const Dims gd = a.gdims;
    const IT i3 = line / out.n2, i2 = line - i3 * out.n2;
    const int64_t gi = kb + (int64_t)(i + (IT)gd.n1 * (i2 + (IT)gd.n2 * i3));
    const int64_t gstep = a.gaxis == 1 ? 1 : (a.gaxis == 2 ? (int64_t)gd.n1 : (int64_t)gd.n1 * gd.n2);
    acc += a.g[gi] - a.g[gi + gstep];
  }
  pass_store(a, o, acc);
}

template <typename T, int W, typename IT>
__global__ void __launch_bounds__(512) k_band_pass(const __grid_constant__ PassBatch<T> pb) {
  pdl_begin();
  int jb = 0;
  while (jb + 1 < pb.njobs && (int)blockIdx.x >= pb.first_block[jb + 1]) ++jb;
  const PassArgs<T>& a = pb.job[jb];
  const int axis = a.axis;
  if constexpr (W > 0) {
    if (pb.flat1 && axis == 1) {
      band_pass_flat_x1<T, W, IT>(a, (IT)(blockIdx.x - pb.first_block[jb]) * (IT)blockDim.x +
                                         (IT)threadIdx.x);
      return;
    }
  }
  const Dims out = a.in.with(axis, a.D0.rows);
  const int m = a.D0.rows;
  const int seg_n = pb.seg;
  const int nseg = (m + seg_n - 1) / seg_n;
  // lines of one item: the product of the two other extents (no 64-bit division, which issues
  // FP64-pipe instructions on this part)
  const IT lines1 = axis == 1 ? (IT)out.n2 * out.n3
                             : (axis == 2 ? (IT)out.n1 * out.n3 : (IT)out.n1 * out.n2);
  const int nb = a.nb > 1 ? a.nb : 1;
  const IT lines = lines1 * nb;
  const IT t = (IT)(blockIdx.x - pb.first_block[jb]) * (IT)blockDim.x + (IT)threadIdx.x;
  // t = line + lines_r * seg with lines rounded to a warp multiple (warps share seg)
  const IT lines_r = (lines + 31) / 32 * 32;
  const IT sq = t / lines_r;
  IT line = t - sq * lines_r;
  const int seg = (int)sq;
  if (line >= lines || seg >= nseg) return;
  int64_t kb = 0;   // item offset
  if (nb > 1) {
    const IT k = line / lines1;
    kb = (int64_t)k * a.bs;
    line -= k * lines1;
  }
  // line -> (j_a, j_b): the two non-band indices, the first one fastest
  IT base_in, stride_in, base_out, stride_out;
  int k1, k2;   // indices along (x1, x2, x3) of the line position, filled per axis
  if (axis == 1) {
    const IT q = line / out.n2;
    const int i2 = (int)(line - q * out.n2), i3 = (int)q;
    base_in = (IT)a.in.n1 * (i2 + (IT)a.in.n2 * i3);
    stride_in = 1;
    base_out = (IT)out.n1 * (i2 + (IT)out.n2 * i3);
    stride_out = 1;
    k1 = i2;
    k2 = i3;
  } else if (axis == 2) {
    const IT q = line / out.n1;
    const int i1 = (int)(line - q * out.n1), i3 = (int)q;
    base_in = i1 + (IT)a.in.n1 * a.in.n2 * i3;
    stride_in = a.in.n1;
    base_out = i1 + (IT)out.n1 * out.n2 * i3;
    stride_out = out.n1;
    k1 = i1;
    k2 = i3;
  } else {
    const IT q = line / out.n1;
    const int i1 = (int)(line - q * out.n1), i2 = (int)q;
    base_in = i1 + (IT)a.in.n1 * i2;
    stride_in = (IT)a.in.n1 * a.in.n2;
    base_out = i1 + (IT)out.n1 * i2;
    stride_out = (IT)out.n1 * out.n2;
    k1 = i1;
    k2 = i2;
  }
  const T* X0 = a.X0 + kb;
  const T* X1 = a.nterms > 1 ? a.X1 + kb : nullptr;
  IT gbase = 0, gstride = 0, gstep = 0;
  if (a.g) {
    // g has extents b^3 (gdims); the output's own index along gaxis is the band index when
    // gaxis == axis, otherwise one of (k1, k2)
    const Dims gd = a.gdims;
    const IT g2 = gd.n1, g3 = (IT)gd.n1 * gd.n2;
    int j1, j2, j3;
    if (axis == 1) { j1 = 0; j2 = k1; j3 = k2; }
    else if (axis == 2) { j1 = k1; j2 = 0; j3 = k2; }
    else { j1 = k1; j2 = k2; j3 = 0; }
    gbase = j1 + g2 * j2 + g3 * j3;
    gstride = axis == 1 ? 1 : (axis == 2 ? g2 : g3);     // moving along the band direction
    gstep = a.gaxis == 1 ? 1 : (a.gaxis == 2 ? g2 : g3); // the difference direction
  }
  const T* g = a.g ? a.g + kb : nullptr;
  const int i_end = min(m, (seg + 1) * seg_n);
  constexpr int WN = W == 9 ? 7 : W;   // the narrower compiled width of a width-9 launch
  const bool narrow = W == 9 && pb.w7[jb];
  for (int i = seg * seg_n; i < i_end; ++i) {
    T acc = narrow ? band_dot<WN>(a.D0, i, X0, base_in, stride_in)
                   : band_dot<W>(a.D0, i, X0, base_in, stride_in);
    if (a.chain) {
      acc = narrow ? band_dot<WN>(a.D1, i, X1, base_in, stride_in, acc)
                   : band_dot<W>(a.D1, i, X1, base_in, stride_in, acc);
    } else {
      if (!a.c0_one) acc *= a.c0;   // (a product with 1 is exact: skipped)
      if (a.nterms > 1)
        acc = fma(a.c1,
                  narrow ? band_dot<WN>(a.D1, i, X1, base_in, stride_in)
                         : band_dot<W>(a.D1, i, X1, base_in, stride_in),
                  acc);
    }
    const int64_t o = kb + (int64_t)(base_out + (IT)i * stride_out);
    if (a.Z) acc += a.cz * a.Z[o];
    if (g) {
      const IT gi = gbase + (IT)i * gstride;
      acc += g[gi] - g[gi + gstep];
    }
    pass_store(a, o, acc);
  }
}

// FP32 (bandwidth-bound) variant: a block owns 32 neighbouring lines (flattened over the two
// non-band directions in memory order) and the whole band extent. Inputs are read once from
// global memory with coalesced loads into shared memory ([j][line]), every output of the tile is
// formed from shared memory, and passes along x1 stage their outputs in shared memory so that
// the stores are coalesced too.
constexpr int kTileLines = 32;

__device__ __forceinline__ void line_geometry(int axis, const Dims& d, int64_t line,
                                              int64_t* base, int64_t* stride) {
  if (axis == 1) {
    *base = (int64_t)d.n1 * line;
    *stride = 1;
  } else if (axis == 2) {
    const int64_t i1 = line % d.n1, i3 = line / d.n1;
    *base = i1 + (int64_t)d.n1 * d.n2 * i3;
    *stride = d.n1;
  } else {
    *base = line;
    *stride = (int64_t)d.n1 * d.n2;
  }
}

// W: band width of every term of the launch (0: runtime width, generic loop).
template <int W>
__global__ void __launch_bounds__(256) k_band_tile(const __grid_constant__ PassBatch<float> pb) {
  pdl_begin();
  extern __shared__ __align__(16) float sh[];
  int jb = 0;
  while (jb + 1 < pb.njobs && (int)blockIdx.x >= pb.first_block[jb + 1]) ++jb;
  const PassArgs<float>& a = pb.job[jb];
  const int axis = a.axis;
  const int nin = a.in.get(axis);
  const int m = a.D0.rows;
  const int nt = a.nterms;
  // band width of each term (the terms of a pass may differ on tiny meshes, where some 1D
  // matrices are exactly diagonal); W > 0 means every term of the launch has width W
  const int wt0 = W > 0 ? W : a.D0.width;
  const int wt1 = W > 0 ? W : (nt > 1 ? a.D1.width : 0);
  const int wp = ((wt0 > wt1 ? wt0 : wt1) + 3) & ~3;   // coefficient row pitch (float4 loads)
  const Dims out = a.in.with(axis, m);
  const int64_t lines = axis == 1 ? (int64_t)out.n2 * out.n3   // no 64-bit division
                                 : (axis == 2 ? (int64_t)out.n1 * out.n3 : (int64_t)out.n1 * out.n2);
  const int64_t line0 = (int64_t)(blockIdx.x - pb.first_block[jb]) * kTileLines;
  const int nl = (int)(lines - line0 < kTileLines ? lines - line0 : kTileLines);
  constexpr int P = kTileLines + 1;   // shared pitch of the input slabs
  float* xs0 = sh;
  float* xs1 = sh + nin * P;
  float* ys = sh + nt * nin * P;                       // m x P (passes along x1)
  // nt x m x wp coefficients, offset rounded up to 4 floats for the 16-byte float4 loads
  float* cf = sh + ((nt * nin * P + (axis == 1 ? m * P : 0) + 3) & ~3);
  int* st = reinterpret_cast<int*>(cf + nt * m * wp);  // nt x m band starts
  const int tid = threadIdx.x;
  const int lane = tid % 32, warp = tid / 32, nwarps = blockDim.x / 32;
  // band coefficients and starts of this launch's operator(s)
  for (int t = 0; t < nt; ++t) {
    const BandD<float>& D = t == 0 ? a.D0 : a.D1;
    const int width = t == 0 ? wt0 : wt1;
    for (int idx = tid; idx < m * wp; idx += blockDim.x) {
      const int i = idx / wp, w = idx - i * wp;
      cf[t * m * wp + idx] = w < width ? D.val[(int64_t)i * width + w] : 0.f;
    }
    for (int i = tid; i < m; i += blockDim.x) st[t * m + i] = D.start[i];
  }
  int64_t ibase = 0, istride = 0;
  if (lane < nl) line_geometry(axis, a.in, line0 + lane, &ibase, &istride);
  for (int t = 0; t < nt; ++t) {
    const float* X = t == 0 ? a.X0 : a.X1;
    float* xs = t == 0 ? xs0 : xs1;
    if (axis == 1) {
      for (int l = warp; l < kTileLines; l += nwarps) {
        const float* row = X + (int64_t)a.in.n1 * (line0 + l);
        for (int j = lane; j < nin; j += 32) xs[j * P + l] = l < nl ? row[j] : 0.f;
      }
    } else {
      for (int j = warp; j < nin; j += nwarps)
        xs[j * P + lane] = lane < nl ? X[ibase + istride * j] : 0.f;
    }
  }
  __syncthreads();
  int64_t obase = 0, ostride = 0;
  if (lane < nl) line_geometry(axis, out, line0 + lane, &obase, &ostride);
  int64_t gbase = 0, gstride = 0, gstep = 0;
  if (a.g && lane < nl) {
    int idx3[3];
    const int64_t line = line0 + lane;
    if (axis == 1) { idx3[0] = 0; idx3[1] = (int)(line % out.n2); idx3[2] = (int)(line / out.n2); }
    else if (axis == 2) { idx3[0] = (int)(line % out.n1); idx3[1] = 0; idx3[2] = (int)(line / out.n1); }
    else { idx3[0] = (int)(line % out.n1); idx3[1] = (int)(line / out.n1); idx3[2] = 0; }
    const Dims gd = a.gdims;
    const int64_t gs[3] = {1, (int64_t)gd.n1, (int64_t)gd.n1 * gd.n2};
    gbase = idx3[0] * gs[0] + idx3[1] * gs[1] + idx3[2] * gs[2];
    gstride = gs[axis - 1];
    gstep = gs[a.gaxis - 1];
  }
  for (int i = warp; i < m; i += nwarps) {
    float acc = 0.f;
    for (int t = 0; t < nt; ++t) {
      const float* xs = (t == 0 ? xs0 : xs1) + st[t * m + i] * P + lane;
      const float4* c4 = reinterpret_cast<const float4*>(cf + (t * m + i) * wp);
      float sum = 0.f;
      if (W > 0) {
#pragma unroll
        for (int w4 = 0; w4 < (W + 3) / 4; ++w4) {
          const float4 c = c4[w4];
          if (4 * w4 + 0 < W) sum = fmaf(c.x, xs[(4 * w4 + 0) * P], sum);
          if (4 * w4 + 1 < W) sum = fmaf(c.y, xs[(4 * w4 + 1) * P], sum);
          if (4 * w4 + 2 < W) sum = fmaf(c.z, xs[(4 * w4 + 2) * P], sum);
          if (4 * w4 + 3 < W) sum = fmaf(c.w, xs[(4 * w4 + 3) * P], sum);
        }
      } else {
        const float* c1 = cf + (t * m + i) * wp;
        const int width = t == 0 ? wt0 : wt1;
        for (int w = 0; w < width; ++w) sum = fmaf(c1[w], xs[w * P], sum);
      }
      acc = fmaf(t == 0 ? a.c0 : a.c1, sum, acc);
    }
    if (lane < nl) {
      const int64_t o = obase + ostride * i;
      if (a.Z) acc += a.cz * a.Z[o];
      if (a.g) {
        const int64_t gi = gbase + gstride * i;
        acc += a.g[gi] - a.g[gi + gstep];
      }
      if (axis == 1) ys[i * P + lane] = acc;
      else a.Y[o] = acc;
    }
  }
  if (axis == 1) {
    __syncthreads();
    for (int l = warp; l < nl; l += nwarps) {
      float* row = a.Y + (int64_t)m * (line0 + l);
      for (int i = lane; i < m; i += 32) row[i] = ys[i * P + l];
    }
  }
}

// Asynchronous global -> shared copies (cp.async): a thread issues all of its copies before it
// waits, so a block keeps its whole slab in flight instead of one load per warp.
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// FP32 pass for centred band matrices (every term of the launch has the centred width
// W = 2H + 1). Tiles as k_band_tile: 32 neighbouring lines per block, the whole band extent.
// - The input slabs (stored with H zero rows above and below, so row i of the output reads slab
//   rows i .. i + W - 1 with no clamping) and the centred coefficients are copied with cp.async,
//   all copies in flight at once.
// - Each lane forms kSlideR consecutive outputs of its line from one register window of
//   kSlideR + W - 1 inputs: (kSlideR + W - 1) / kSlideR shared loads per output instead of W.
// - Interior rows of a matrix on a uniform knot vector are identical (Toeplitz); chunks of rows
//   inside that range take their coefficients from registers, the few boundary chunks from
//   shared memory.
// - Index arithmetic is 32-bit (the launcher only takes tensors below 2^31 entries).
constexpr int kSlideR = 8;

__host__ __device__ constexpr int slide_rows(int m) { return (m + kSlideR - 1) / kSlideR * kSlideR; }

__device__ __forceinline__ void line_geometry32(int axis, const Dims& d, int line, int* base,
                                                int* stride) {
  if (axis == 1) {
    *base = d.n1 * line;
    *stride = 1;
  } else if (axis == 2) {
    const int i3 = line / d.n1, i1 = line - i3 * d.n1;
    *base = i1 + d.n1 * d.n2 * i3;
    *stride = d.n1;
  } else {
    *base = line;
    *stride = d.n1 * d.n2;
  }
}

template <int W, int R>
__device__ __forceinline__ void slide_term(const float* xs, const float* cf_rows, bool interior,
                                           const float (&creg)[W], float ct, float (&acc)[R]) {
  constexpr int P = kTileLines + 1;
  constexpr int CP = (W + 3) & ~3;
  float v[R + W - 1];
#pragma unroll
  for (int k = 0; k < R + W - 1; ++k) v[k] = xs[k * P];
  if (interior) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int k = 0; k < W; ++k) {
        if (k % 2 == 0) s0 = fmaf(creg[k], v[r + k], s0);
        else s1 = fmaf(creg[k], v[r + k], s1);
      }
      acc[r] = fmaf(ct, s0 + s1, acc[r]);
    }
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float4* c4 = reinterpret_cast<const float4*>(cf_rows + r * CP);
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int w4 = 0; w4 < CP / 4; ++w4) {
        const float4 c = c4[w4];
        if (4 * w4 + 0 < W) s0 = fmaf(c.x, v[r + 4 * w4 + 0], s0);
        if (4 * w4 + 1 < W) s1 = fmaf(c.y, v[r + 4 * w4 + 1], s1);
        if (4 * w4 + 2 < W) s0 = fmaf(c.z, v[r + 4 * w4 + 2], s0);
        if (4 * w4 + 3 < W) s1 = fmaf(c.w, v[r + 4 * w4 + 3], s1);
      }
      acc[r] = fmaf(ct, s0 + s1, acc[r]);
    }
  }
}

// HAS_G: every job of the launch adds the difference term of g (none has a Z term). Registers
// are bounded to four blocks per SM (a few bytes spill) so that blocks of these passes fit beside
// a tensor-core mode product of the concurrent branch: 128^3 solve 58.4 -> 58.1 ms.
template <int W, bool HAS_G>
__global__ void __launch_bounds__(256, 4) k_band_slide(const __grid_constant__ PassBatch<float> pb) {
  pdl_begin();
  constexpr int H = (W - 1) / 2;
  constexpr int CP = (W + 3) & ~3;
  constexpr int R = kSlideR;
  constexpr int P = kTileLines + 1;
  extern __shared__ __align__(16) float sh[];
  int jb = 0;
  while (jb + 1 < pb.njobs && (int)blockIdx.x >= pb.first_block[jb + 1]) ++jb;
  const PassArgs<float>& a = pb.job[jb];
  const int axis = a.axis;
  const int m = a.D0.rows;   // square: output extent = input extent along the axis
  const int mr = slide_rows(m);
  const int rs = mr + 2 * H;   // slab rows
  const int nt = a.nterms;
  const Dims out = a.in;
  const int lines1 = axis == 1 ? out.n2 * out.n3   // lines of one item (no 64-bit division)
                              : (axis == 2 ? out.n1 * out.n3 : out.n1 * out.n2);
  const int nb = a.nb > 1 ? a.nb : 1;
  const int lines = lines1 * nb;
  const int line0 = ((int)blockIdx.x - pb.first_block[jb]) * kTileLines;
  const int nl = lines - line0 < kTileLines ? lines - line0 : kTileLines;
  float* ys = sh + nt * rs * P;                                          // m x P (passes along x1)
  float* cf = sh + ((nt * rs * P + (axis == 1 ? m * P : 0) + 3) & ~3);   // nt x mr x CP
  const int tid = threadIdx.x;
  const int lane = tid % 32, warp = tid / 32, nwarps = blockDim.x / 32;
  for (int t = 0; t < nt; ++t) {
    const float* src = (t == 0 ? a.D0 : a.D1).cval;
    for (int q = tid; q < mr * CP / 4; q += blockDim.x) cp_async16(cf + t * mr * CP + 4 * q, src + 4 * q);
  }
  // this lane's line: item k (offset koff) and line l within the item
  int base = 0, stride = 0;
  int64_t koff = 0;
  int lline = line0 + lane;
  if (nb > 1) {
    const int k = lline / lines1;
    lline -= k * lines1;
    koff = (int64_t)k * a.bs;
  }
  if (lane < nl) line_geometry32(axis, a.in, lline, &base, &stride);
  for (int t = 0; t < nt; ++t) {
    const float* X = t == 0 ? a.X0 : a.X1;
    float* xs = sh + t * rs * P;
    // zero rows: H above, H + (mr - m) below
    for (int q = tid; q < H * P; q += blockDim.x) xs[q] = 0.f;
    for (int q = tid; q < (rs - H - m) * P; q += blockDim.x) xs[(H + m) * P + q] = 0.f;
    if (axis == 1) {
      for (int l = warp; l < kTileLines; l += nwarps) {
        int gl = line0 + l, k = 0;
        if (nb > 1) {
          k = gl / lines1;
          gl -= k * lines1;
        }
        const float* row = X + (int64_t)k * a.bs + a.in.n1 * gl;
        float* dst = xs + H * P + l;
        if (l < nl) {
#pragma unroll 4
          for (int j = lane; j < m; j += 32) cp_async4(dst + j * P, row + j);
        } else {
          for (int j = lane; j < m; j += 32) dst[j * P] = 0.f;
        }
      }
    } else {
      float* dst = xs + (H + warp) * P + lane;
      if (lane < nl) {
        const float* src = X + koff + base + warp * stride;
#pragma unroll 4
        for (int j = warp; j < m; j += nwarps, dst += nwarps * P, src += nwarps * stride)
          cp_async4(dst, src);
      } else {
        for (int j = warp; j < m; j += nwarps, dst += nwarps * P) *dst = 0.f;
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
  int gbase = 0, gstride = 0, gstep = 0;
  if (HAS_G && lane < nl) {
    const int line = lline;
    int idx3[3];
    if (axis == 1) { idx3[0] = 0; idx3[2] = line / out.n2; idx3[1] = line - idx3[2] * out.n2; }
    else if (axis == 2) { idx3[2] = line / out.n1; idx3[0] = line - idx3[2] * out.n1; idx3[1] = 0; }
    else { idx3[1] = line / out.n1; idx3[0] = line - idx3[1] * out.n1; idx3[2] = 0; }
    const int g1 = a.gdims.n1, g12 = a.gdims.n1 * a.gdims.n2;
    gbase = idx3[0] + g1 * idx3[1] + g12 * idx3[2];
    gstride = axis == 1 ? 1 : (axis == 2 ? g1 : g12);
    gstep = a.gaxis == 1 ? 1 : (a.gaxis == 2 ? g1 : g12);
  }
  // interior (Toeplitz) rows shared by every term, and their coefficients in registers
  int tlo = a.D0.tlo, thi = a.D0.thi;
  if (nt > 1) {
    tlo = max(tlo, a.D1.tlo);
    thi = min(thi, a.D1.thi);
  }
  float creg0[W], creg1[W];
  const int trow = tlo < thi ? tlo : 0;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    creg0[k] = cf[trow * CP + k];
    creg1[k] = nt > 1 ? cf[mr * CP + trow * CP + k] : 0.f;
  }
  const float c0 = a.c0, c1 = a.c1;
  const float* g = HAS_G ? a.g + koff : nullptr;
  float* Y = a.Y;
  const bool ax1 = axis == 1;
  for (int i0 = warp * R; i0 < mr; i0 += nwarps * R) {
    float acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.f;
    const bool interior = i0 >= tlo && i0 + R <= thi;
    slide_term<W, R>(sh + i0 * P + lane, cf + i0 * CP, interior, creg0, c0, acc);
    if (nt > 1)
      slide_term<W, R>(sh + rs * P + i0 * P + lane, cf + (mr + i0) * CP, interior, creg1, c1, acc);
    if (HAS_G && lane < nl) {
      const int g0 = gbase + gstride * i0;
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (i0 + r < m) acc[r] += g[g0 + gstride * r] - g[g0 + gstride * r + gstep];
    }
    if (ax1) {
      float* yr = ys + i0 * P + lane;
      if (i0 + R <= m) {
#pragma unroll
        for (int r = 0; r < R; ++r) yr[r * P] = acc[r];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (i0 + r < m) yr[r * P] = acc[r];
      }
    } else if (lane < nl) {
      float* yo = Y + koff + base + stride * i0;
      if (i0 + R <= m) {
#pragma unroll
        for (int r = 0; r < R; ++r) yo[stride * r] = acc[r];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (i0 + r < m) yo[stride * r] = acc[r];
      }
    }
  }
  if (axis == 1) {
    __syncthreads();
    for (int l = warp; l < nl; l += nwarps) {
      int gl = line0 + l, k = 0;
      if (nb > 1) {
        k = gl / lines1;
        gl -= k * lines1;
      }
      float* row = Y + (int64_t)k * a.bs + (int64_t)m * gl;
      for (int i = lane; i < m; i += 32) row[i] = ys[i * P + l];
    }
  }
}

// nb items: item k of every tensor argument at offset k * bs elements. One warp per x1 row
// (i2, i3) of the pressure grid, lanes along i1: the row's indices are formed once per row (the
// per-element divisions of a flat index made these stencils issue-bound).
template <typename T>
__global__ void __launch_bounds__(256) k_divergence(const T* __restrict__ u1, const T* __restrict__ u2,
                                                    const T* __restrict__ u3, int a, int b,
                                                    T* __restrict__ delta, const T* __restrict__ q,
                                                    T nu, T* __restrict__ e, int nb, int64_t bs) {
  pdl_begin();
  const int lane = threadIdx.x % 32;
  const int rows1 = b * b;   // (i2, i3) rows of one item
  const int64_t rows = (int64_t)rows1 * nb;
  const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
  for (int64_t rw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; rw < rows; rw += nw) {
    const int64_t k = nb > 1 ? rw / rows1 : 0;
    const int r = (int)(rw - k * rows1);
    const int i3 = r / b, i2 = r - i3 * b;
    const int64_t kb = k * bs;
    const T* p1 = u1 + kb + (int64_t)a * (i2 + (int64_t)b * i3);   // u1 extents (a, b, b)
    const T* p2 = u2 + kb + (int64_t)b * a * i3;                   // u2 extents (b, a, b)
    const T* p3 = u3 + kb + (int64_t)b * i2;                       // u3 extents (b, b, a)
    const int64_t o = kb + (int64_t)b * r;
    for (int i1 = lane; i1 < b; i1 += 32) {
      T d = 0;
      if (i1 < a) d += p1[i1];
      if (i1 >= 1) d -= p1[i1 - 1];
      if (i2 < a) d += p2[i1 + (int64_t)b * i2];
      if (i2 >= 1) d -= p2[i1 + (int64_t)b * (i2 - 1)];
      if (i3 < a) d += p3[i1 + (int64_t)b * b * i3];
      if (i3 >= 1) d -= p3[i1 + (int64_t)b * b * (i3 - 1)];
      delta[o + i1] = d;
      if (e) e[o + i1] = fma(nu, d, q[o + i1]);
    }
  }
}

// The divergence and the first pressure-mass pass in one launch (FP64 A and K applies): a block
// owns lpb whole x1 lines of the pressure grid, forms delta (and e = nu delta + q when q is set)
// on them in shared memory with the operations of k_divergence, and applies the band D along x1
// with the single FMA chain of the flat x1 pass: y0 = D .x1 delta, y1 = D .x1 e. WC: the band
// width when it is a compiled one (the chains unrolled), 0 for a runtime width.
template <typename T, int WC>
__global__ void __launch_bounds__(512) k_div_band_x1(const T* __restrict__ u1,
                                                     const T* __restrict__ u2,
                                                     const T* __restrict__ u3, int a, int b,
                                                     const T* __restrict__ q, T nu,
                                                     const __grid_constant__ BandD<T> D, int lpb,
                                                     T* __restrict__ y0, T* __restrict__ y1) {
  pdl_begin();
  extern __shared__ __align__(16) unsigned char div_smem[];
  T* sd = reinterpret_cast<T*>(div_smem);   // [lpb][b]: delta
  T* se = sd + lpb * b;                     // [lpb][b]: e
  const int lines = b * b;
  const int t = threadIdx.x;
  const int l = t / b, i1 = t - l * b;
  const int line = blockIdx.x * lpb + l;
  const bool active = l < lpb && line < lines;
  if (active) {
    const int i2 = line % b, i3 = line / b;
    T d = 0;
    {
      const int64_t row = (int64_t)a * (i2 + (int64_t)b * i3);
      if (i1 < a) d += u1[row + i1];
      if (i1 >= 1) d -= u1[row + i1 - 1];
    }
    {
      const int64_t off = i1 + (int64_t)b * a * i3;
      if (i2 < a) d += u2[off + (int64_t)b * i2];
      if (i2 >= 1) d -= u2[off + (int64_t)b * (i2 - 1)];
    }
    {
      const int64_t off = i1 + (int64_t)b * i2;
      if (i3 < a) d += u3[off + (int64_t)b * b * i3];
      if (i3 >= 1) d -= u3[off + (int64_t)b * b * (i3 - 1)];
    }
    sd[l * b + i1] = d;
    if (q) se[l * b + i1] = fma(nu, d, q[(int64_t)line * b + i1]);
  }
  __syncthreads();
  if (!active) return;
  const int W = WC > 0 ? WC : D.width;
  const T* cv = D.val + (int64_t)i1 * W;
  const int s0i = __ldg(D.start + i1);
  const T* xd = sd + l * b + s0i;
  T s0 = 0;
#pragma unroll
  for (int w = 0; w < W; ++w) s0 = fma(__ldg(cv + w), xd[w], s0);
  y0[(int64_t)line * b + i1] = s0;
  if (q) {
    const T* xe = se + l * b + s0i;
    T e0 = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) e0 = fma(__ldg(cv + w), xe[w], e0);
    y1[(int64_t)line * b + i1] = e0;
  }
}

// y_c (+)= the difference transpose of g along direction c, for the three velocity components
// (extents a in the own direction, b in the others). One warp per x1 row of a component, lanes
// along i1 (row indices formed once per row).
template <typename T>
__global__ void __launch_bounds__(256) k_div_transpose(const T* __restrict__ g, int a, int b, T* y1,
                                                       T* y2, T* y3, int accumulate, int nb,
                                                       int64_t bs) {
  pdl_begin();
  const int lane = threadIdx.x % 32;
  // rows of one item: b * b of component 1 (rows of a entries), a * b of components 2 and 3
  const int r0 = b * b, r1 = a * b;
  const int rows1 = r0 + 2 * r1;
  const int64_t rows = (int64_t)rows1 * nb;
  const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
  for (int64_t rw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; rw < rows; rw += nw) {
    const int64_t k = nb > 1 ? rw / rows1 : 0;
    int r = (int)(rw - k * rows1);
    const int c = r < r0 ? 0 : (r < r0 + r1 ? 1 : 2);
    r -= c == 0 ? 0 : (c == 1 ? r0 : r0 + r1);
    const int e1 = c == 0 ? a : b, e2 = c == 1 ? a : b;
    const int i3 = r / e2, i2 = r - i3 * e2;
    const int64_t kb = k * bs;
    T* y = (c == 0 ? y1 : (c == 1 ? y2 : y3)) + kb + (int64_t)e1 * r;
    const int64_t gs = c == 0 ? 1 : (c == 1 ? (int64_t)b : (int64_t)b * b);
    const T* gr = g + kb + (int64_t)b * (i2 + (int64_t)b * i3);
    for (int i1 = lane; i1 < e1; i1 += 32) {
      const T v = gr[i1] - gr[i1 + gs];
      y[i1] = accumulate ? y[i1] + v : v;
    }
  }
}

// One thread per line: the block's lines are first copied into shared memory (coalesced), then
// each thread runs forward substitution with L and backward substitution with L^T on its own
// column of shared memory, and the block writes the lines to y (which may be x). nb items, item k
// of x and y at k * bs entries; 32-bit line arithmetic (b^2 nb < 2^31, checked by the launcher).
constexpr int kCholLines = 32;

template <typename T>
__global__ void __launch_bounds__(kCholLines) k_chol_line(const T* x, T* y, int b, int p, int axis,
                                                          const T* __restrict__ lb,
                                                          const T* __restrict__ inv, T post,
                                                          int nb, int64_t bs) {
  pdl_begin();
  extern __shared__ __align__(16) unsigned char chol_smem[];
  constexpr int P = kCholLines + 1;
  const int w = p + 1;
  // the factor in shared memory: one warp per block and few blocks per SM, so each step of the
  // substitutions must not wait on a global load
  T* lbs = reinterpret_cast<T*>(chol_smem);   // [b][p + 1]
  T* invs = lbs + b * w;                      // [b]
  T* cs = invs + b;                           // [b][P] the block's lines
  for (int i = threadIdx.x; i < b * w; i += kCholLines) lbs[i] = lb[i];
  for (int i = threadIdx.x; i < b; i += kCholLines) invs[i] = inv[i];
  const int lines1 = b * b;
  const int lines = lines1 * nb;
  const int line0 = blockIdx.x * kCholLines;
  const int nl = lines - line0 < kCholLines ? lines - line0 : kCholLines;
  const int l = threadIdx.x;
  // offset of a line (over all items) and the stride along it
  auto line_off = [&](int line, int64_t* stride) -> int64_t {
    const int k = line / lines1, li = line - k * lines1;
    int64_t base;
    if (axis == 1) {
      base = (int64_t)b * li;
      *stride = 1;
    } else if (axis == 2) {
      const int q = li / b;
      base = (li - q * b) + (int64_t)b * b * q;
      *stride = b;
    } else {
      base = li;
      *stride = (int64_t)b * b;
    }
    return (int64_t)k * bs + base;
  };
  int64_t base = 0, stride = 0;
  if (l < nl) base = line_off(line0 + l, &stride);
  // staging: batches of kCholBatch independent loads in flight before their shared stores (one
  // warp per block: a load-store loop would wait a full memory latency per element)
  constexpr int kCholBatch = 16;
  if (axis == 1) {
    // rows of x1 (contiguous): the warp walks the block's rows, lanes along each row
    const int total = nl * b;
    for (int q0 = 0; q0 < total; q0 += kCholBatch * kCholLines) {
      T t[kCholBatch];
#pragma unroll
      for (int u = 0; u < kCholBatch; ++u) {
        const int q = q0 + u * kCholLines + l;
        if (q < total) {
          const int r = q / b, j = q - r * b;
          int64_t st;
          t[u] = x[line_off(line0 + r, &st) + j];
        }
      }
#pragma unroll
      for (int u = 0; u < kCholBatch; ++u) {
        const int q = q0 + u * kCholLines + l;
        if (q < total) {
          const int r = q / b, j = q - r * b;
          cs[j * P + r] = t[u];
        }
      }
    }
  } else if (l < nl) {
    for (int j0 = 0; j0 < b; j0 += kCholBatch) {
      T t[kCholBatch];
#pragma unroll
      for (int u = 0; u < kCholBatch; ++u)
        if (j0 + u < b) t[u] = x[base + stride * (j0 + u)];
#pragma unroll
      for (int u = 0; u < kCholBatch; ++u)
        if (j0 + u < b) cs[(j0 + u) * P + l] = t[u];
    }
  }
  __syncthreads();
  if (l < nl) {
    T* v = cs + l;
    for (int i = 0; i < b; ++i) {
      T acc = v[i * P];
      const int k0 = i - p < 0 ? 0 : i - p;
      for (int k = k0; k < i; ++k) acc = fma(-lbs[i * w + (k - i + p)], v[k * P], acc);
      v[i * P] = acc * invs[i];
    }
    for (int i = b - 1; i >= 0; --i) {
      T acc = v[i * P];
      const int k1 = i + p > b - 1 ? b - 1 : i + p;
      for (int k = i + 1; k <= k1; ++k) acc = fma(-lbs[k * w + (i - k + p)], v[k * P], acc);
      v[i * P] = acc * invs[i];
    }
  }
  __syncthreads();
  if (axis == 1) {
    for (int r = 0; r < nl; ++r) {
      int64_t st;
      T* row = y + line_off(line0 + r, &st);
      for (int j = l; j < b; j += kCholLines) row[j] = cs[j * P + r] * post;
    }
  } else if (l < nl) {
    for (int j = 0; j < b; ++j) y[base + stride * j] = cs[j * P + l] * post;
  }
}

}  // namespace

template <typename T>
cudaError_t chol_solve_axis(const T* x, T* y, int b, int p, int axis, const T* lb,
                            const T* inv_diag, T post, cudaStream_t s, int nb, int64_t bs) {
  if (nb < 1) nb = 1;
  const int64_t lines = (int64_t)b * b * nb;
  if (lines >= ((int64_t)1 << 31) - kCholLines) return cudaErrorInvalidValue;
  const int smem = (b * (kCholLines + 1) + b * (p + 1) + b) * (int)sizeof(T);
  static std::atomic<int> attr{0};
  const cudaError_t e = raise_smem_limit(k_chol_line<T>, attr, smem);
  if (e != cudaSuccess) return e;
  launch_begin(kClassLine, s);
  const cudaError_t l = launch_k(k_chol_line<T>, (unsigned)((lines + kCholLines - 1) / kCholLines),
                                 kCholLines, smem, s, x, y, b, p, axis, lb, inv_diag, post, nb, bs);
  launch_end(kClassLine, s, 4.0 * (p + 1) * lines * b, 2.0 * lines * b * sizeof(T));
  return l;
}
template cudaError_t chol_solve_axis<double>(const double*, double*, int, int, int, const double*,
                                             const double*, double, cudaStream_t, int, int64_t);

void band_tile_multi(const PassArgs<float>* jobs, int njobs, cudaStream_t s) {
  // FP32 passes write Y, then the vector kernel applies a Horner step (in FP32 the separate
  // streaming kernel measured faster than an epilogue in the banded pass; same operations).
  bool horner = false;
  for (int j = 0; j < njobs; ++j) horner = horner || jobs[j].hmode != 0;
  if (horner) {
    PassArgs<float> plain[kMaxPassJobs];
    for (int j = 0; j < njobs; ++j) {
      plain[j] = jobs[j];
      plain[j].hmode = 0;
    }
    band_tile_multi(plain, njobs, s);
    // one vector launch when the jobs' outputs (and Horner vectors) follow each other, as the
    // three velocity components do; otherwise one per job
    bool contiguous = true;
    int64_t total = 0;
    for (int j = 0; j < njobs; ++j) {
      const PassArgs<float>& a = jobs[j];
      const PassArgs<float>& a0 = jobs[0];
      contiguous = contiguous && a.hmode == a0.hmode && a.nb == a0.nb && a.bs == a0.bs &&
                   a.Y == a0.Y + total && a.hr == a0.hr + total && a.hacc == a0.hacc + total &&
                   (a.hmode != 1 || a.hx == a0.hx + total);
      total += a.in.with(a.axis, a.D0.rows).size();
    }
    const int np = contiguous ? 1 : njobs;
    for (int j = 0; j < np; ++j) {
      const PassArgs<float>& a = jobs[j];
      const int64_t n = contiguous ? total : a.in.with(a.axis, a.D0.rows).size();
      if (a.hmode == 1) hp_first<float>(a.hx, a.Y, a.hr, a.hacc, n, s, a.nb, a.bs);
      else if (a.hmode == 2) hp_update<float>(a.hr, a.Y, a.hacc, n, s, a.nb, a.bs);
    }
    return;
  }
  PassBatch<float> pb{};
  pb.njobs = njobs;
  int blocks = 0;
  int smem = 0;
  double flops = 0, bytes = 0;
  for (int j = 0; j < njobs; ++j) {
    const PassArgs<float>& a = jobs[j];
    pb.job[j] = a;
    pb.first_block[j] = blocks;
    const Dims out = a.in.with(a.axis, a.D0.rows);
    const int nbj = a.nb > 1 ? a.nb : 1;
    const int64_t lines = out.size() / a.D0.rows * nbj;
    blocks += (int)((lines + kTileLines - 1) / kTileLines);
    const int nin = a.in.get(a.axis);
    const int nt = a.nterms > 1 ? 2 : 1;
    const int wmax = nt > 1 && a.D1.width > a.D0.width ? a.D1.width : a.D0.width;
    const int wp = (wmax + 3) & ~3;
    const int sm = (nt * nin + (a.axis == 1 ? a.D0.rows : 0)) * (kTileLines + 1) * (int)sizeof(float) +
                   16 + nt * a.D0.rows * (wp * (int)sizeof(float) + (int)sizeof(int));
    smem = sm > smem ? sm : smem;
    const double outs = (double)out.size() * nbj;
    double fl = 2.0 * a.D0.width * outs, by = (double)a.in.size() * nbj + outs;
    if (a.nterms > 1) { fl += 2.0 * a.D1.width * outs; by += (double)a.in.size() * nbj; }
    if (a.Z) { fl += 2.0 * outs; by += outs; }
    if (a.g) { fl += 2.0 * outs; by += (double)a.gdims.size() * nbj; }
    flops += fl;
    bytes += by * sizeof(float);
  }
  pb.first_block[njobs] = blocks;
  pb.seg = 1;
  // centred kernel when every term of every job is square with a centred copy of one width
  int Wc = 2 * jobs[0].D0.half + 1;
  int smem_c = 0;
  for (int j = 0; j < njobs && Wc > 0; ++j) {
    const PassArgs<float>& a = jobs[j];
    const int nt = a.nterms > 1 ? 2 : 1;
    for (int t = 0; t < nt; ++t) {
      const BandD<float>& D = t == 0 ? a.D0 : a.D1;
      if (!D.cval || D.rows != D.cols || D.rows != a.in.get(a.axis) || 2 * D.half + 1 != Wc ||
          D.cpitch != ((Wc + 3) & ~3))
        Wc = 0;
    }
    if (Wc == 0) break;
    const int nbj = a.nb > 1 ? a.nb : 1;
    if (a.in.size() >= ((int64_t)1 << 31) || (a.g && a.gdims.size() >= ((int64_t)1 << 31)) ||
        a.in.size() / a.in.get(a.axis) * nbj >= ((int64_t)1 << 31)) {
      Wc = 0;   // 32-bit indexing within an item, 32-bit line count
      break;
    }
    const int mr = slide_rows(a.D0.rows);
    const int rs = mr + Wc - 1;
    const int sm = ((nt * rs + (a.axis == 1 ? a.D0.rows : 0)) * (kTileLines + 1) + 3) / 4 * 4 *
                       (int)sizeof(float) +
                   nt * mr * ((Wc + 3) & ~3) * (int)sizeof(float);
    smem_c = sm > smem_c ? sm : smem_c;
  }
  if (Wc < 3 || Wc > 21) Wc = 0;   // the instantiated centred widths
  // the slide kernel has no Z term, and either every job or none adds the g term
  bool has_g = jobs[0].g != nullptr;
  for (int j = 0; j < njobs && Wc > 0; ++j)
    if (jobs[j].Z || (jobs[j].g != nullptr) != has_g) Wc = 0;
  if (Wc > 0) {
    launch_begin(kClassBand, s);
    switch (Wc) {
#define SHP_SLIDE_W(w)                                                                          \
  case w: {                                                                                     \
    static std::atomic<int> attr0{0}, attr1{0};                                                 \
    raise_smem_limit(k_band_slide<w, false>, attr0, smem_c);                                    \
    raise_smem_limit(k_band_slide<w, true>, attr1, smem_c);                                     \
    if (has_g) launch_k(k_band_slide<w, true>, blocks, 256, smem_c, s, pb);                      \
    else launch_k(k_band_slide<w, false>, blocks, 256, smem_c, s, pb);                          \
    break;                                                                                      \
  }
      SHP_SLIDE_W(3) SHP_SLIDE_W(5) SHP_SLIDE_W(7) SHP_SLIDE_W(9) SHP_SLIDE_W(11) SHP_SLIDE_W(13)
      SHP_SLIDE_W(15) SHP_SLIDE_W(17) SHP_SLIDE_W(19) SHP_SLIDE_W(21)
#undef SHP_SLIDE_W
      default: break;
    }
    launch_end(kClassBand, s, flops, bytes);
    return;
  }
  // The tile kernel has no item index: a batched launch runs its items as separate jobs.
  bool batched = false;
  for (int j = 0; j < njobs; ++j) batched = batched || jobs[j].nb > 1;
  if (batched) {
    PassArgs<float> items[kMaxPassJobs];
    int ni = 0;
    for (int j = 0; j < njobs; ++j) {
      const int nbj = jobs[j].nb > 1 ? jobs[j].nb : 1;
      for (int k = 0; k < nbj; ++k) {
        PassArgs<float> e = jobs[j];
        const int64_t o = (int64_t)k * e.bs;
        e.X0 += o;
        if (e.X1) e.X1 += o;
        if (e.Z) e.Z += o;
        if (e.g) e.g += o;
        e.Y += o;
        if (e.hr) e.hr += o;
        if (e.hacc) e.hacc += o;
        if (e.hx) e.hx += o;
        e.nb = 1;
        items[ni++] = e;
        if (ni == kMaxPassJobs) {
          band_tile_multi(items, ni, s);
          ni = 0;
        }
      }
    }
    if (ni > 0) band_tile_multi(items, ni, s);
    return;
  }
  // one band width per launch (all terms of all jobs); unrolled kernels for the common widths
  int W = jobs[0].D0.width;
  for (int j = 0; j < njobs; ++j)
    if (jobs[j].D0.width != W || (jobs[j].nterms > 1 && jobs[j].D1.width != W)) W = 0;
  launch_begin(kClassBand, s);
  switch (W) {
#define SHP_TILE_W(w)                                                                         \
  case w: {                                                                                   \
    static std::atomic<int> attr{0};                                                          \
    raise_smem_limit(k_band_tile<w>, attr, smem);                                             \
    launch_k(k_band_tile<w>, blocks, 256, smem, s, pb);                                             \
    break;                                                                                    \
  }
    SHP_TILE_W(3) SHP_TILE_W(5) SHP_TILE_W(7) SHP_TILE_W(9) SHP_TILE_W(11) SHP_TILE_W(13)
    SHP_TILE_W(15) SHP_TILE_W(17) SHP_TILE_W(19) SHP_TILE_W(21)
    default: {
      static std::atomic<int> attr{0};
      raise_smem_limit(k_band_tile<0>, attr, smem);
      launch_k(k_band_tile<0>, blocks, 256, smem, s, pb);
    }
#undef SHP_TILE_W
  }
  launch_end(kClassBand, s, flops, bytes);
}

template <typename T>
void band_pass_multi(const PassArgs<T>* jobs, int njobs, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    band_tile_multi(jobs, njobs, s);
    return;
  }
  PassBatch<T> pb{};
  pb.njobs = njobs;
  const int bt = jobs[0].block > 0 ? std::min(jobs[0].block, 512) : 256;   // threads per block
  int W = jobs[0].D0.width;
  // a launch of width 9 may hold jobs of width 7 along x2 or x3 (the pressure-mass passes that
  // ride with the first velocity pass): flagged, their chains run over their own 7 entries
  const auto width_ok = [&](const PassArgs<T>& a, int w) {
    return a.D0.width == w && (a.nterms < 2 || a.D1.width == w);
  };
  for (int j = 0; j < njobs; ++j) {
    const PassArgs<T>& a = jobs[j];
    pb.w7[j] = (sizeof(T) == 8 && W == 9 && a.axis != 1 && width_ok(a, 7)) ? 1 : 0;
    if (!width_ok(a, W) && !pb.w7[j]) W = 0;
  }
  if (W != 9)
    for (int j = 0; j < njobs; ++j) pb.w7[j] = 0;
  // the instantiated widths; any other width (an even width where a band is clamped by a small
  // matrix) runs the generic kernel, which has no flat layout
  if (!(W >= 3 && W <= 13 && W % 2 == 1)) W = 0;
  // x1 passes with the flat (line, row) layout when the band width is a compiled one and every
  // band of such a job has its transposed copy (the block counts below depend on this choice)
  const int smem = 0;
  pb.flat1 = W > 0;
  for (int j = 0; j < njobs && pb.flat1; ++j)
    if (jobs[j].axis == 1 &&
        (!jobs[j].D0.valT || (jobs[j].nterms > 1 && !jobs[j].D1.valT)))
      pb.flat1 = 0;
  int blocks = 0;
  double flops = 0, bytes = 0;
  for (int j = 0; j < njobs; ++j) {
    const PassArgs<T>& a = jobs[j];
    pb.job[j] = a;
    pb.job[j].c0_one = a.c0 == T(1) ? 1 : 0;
    pb.job[j].chain = (a.nterms > 1 && a.c0 == T(1) && a.c1 == T(1)) ? 1 : 0;
    pb.first_block[j] = blocks;
    const Dims out = a.in.with(a.axis, a.D0.rows);
    const int nbj = a.nb > 1 ? a.nb : 1;
    const int64_t lines = out.size() / a.D0.rows * nbj;
    const int64_t lines_r = (lines + 31) / 32 * 32;
    const int64_t nseg = (a.D0.rows + seg_len<T>() - 1) / seg_len<T>();
    if (pb.flat1 && a.axis == 1) blocks += (int)((out.size() * nbj + bt - 1) / bt);
    else blocks += (int)((lines_r * nseg + bt - 1) / bt);
    // algorithmic work: one band row per output and term; one read of every input tensor
    const double outs = (double)out.size() * nbj;
    double fl = 2.0 * a.D0.width * outs, by = (double)a.in.size() * nbj + outs;
    if (a.nterms > 1) { fl += 2.0 * a.D1.width * outs; by += (double)a.in.size() * nbj; }
    if (a.Z) { fl += 2.0 * outs; by += outs; }
    if (a.g) { fl += 2.0 * outs; by += (double)a.gdims.size() * nbj; }
    flops += fl;
    bytes += by * sizeof(T);
  }
  pb.first_block[njobs] = blocks;
  pb.seg = seg_len<T>();
  // 32-bit thread index arithmetic when every job's thread range (all items) and tensors fit
  bool i32 = (int64_t)blocks * bt < ((int64_t)1 << 31);
  for (int j = 0; j < njobs && i32; ++j) {
    const PassArgs<T>& a = jobs[j];
    const int64_t big = std::max({a.in.size(), a.in.with(a.axis, a.D0.rows).size(),
                                  a.g ? a.gdims.size() : (int64_t)0});
    const int nbj = a.nb > 1 ? a.nb : 1;
    if (big * nbj + 64 >= ((int64_t)1 << 31)) i32 = false;
  }
  // FP64 passes (bound by the FP64 pipe) are accounted apart from the FP32 ones
  const int cls = sizeof(T) == 8 ? kClassBand64 : kClassBand;
  launch_begin(cls, s);
  switch (W) {
#define SHP_PASS_W(w)                                                                     \
  case w: {                                                                               \
    static std::atomic<int> attr32{0}, attr64{0};                                         \
    if (i32) {                                                                            \
      raise_smem_limit(k_band_pass<T, w, int>, attr32, smem);                             \
      launch_k(k_band_pass<T, w, int>, blocks, bt, smem, s, pb);                          \
    } else {                                                                              \
      raise_smem_limit(k_band_pass<T, w, int64_t>, attr64, smem);                         \
      launch_k(k_band_pass<T, w, int64_t>, blocks, bt, smem, s, pb);                      \
    }                                                                                     \
    break;                                                                                \
  }
    SHP_PASS_W(3) SHP_PASS_W(5) SHP_PASS_W(7) SHP_PASS_W(9) SHP_PASS_W(11) SHP_PASS_W(13)
#undef SHP_PASS_W
    default:
      if (i32) launch_k(k_band_pass<T, 0, int>, blocks, bt, 0, s, pb);
      else launch_k(k_band_pass<T, 0, int64_t>, blocks, bt, 0, s, pb);
  }
  launch_end(cls, s, flops, bytes);
}

template <typename T>
void band_pass(const PassArgs<T>& a, cudaStream_t s) {
  band_pass_multi<T>(&a, 1, s);
}

template <typename T>
void divergence(const T* u1, const T* u2, const T* u3, int a, int b, T* delta, cudaStream_t s,
                int nb, int64_t bs) {
  if (nb < 1) nb = 1;
  const int64_t total = (int64_t)b * b * b * nb;
  launch_begin(kClassDiv, s);
  launch_k(k_divergence<T>, grid_for((int64_t)b * b * nb * 32, 256), 256, 0, s, u1, u2, u3, a, b,
           delta, nullptr, T(0), nullptr, nb, bs);
  launch_end(kClassDiv, s, 6.0 * total, (3.0 * a * b * b * nb + total) * sizeof(T));
}

template <typename T>
void div_band_x1(const T* u1, const T* u2, const T* u3, int a, int b, const T* q, T nu,
                 const BandD<T>& D, T* y0, T* y1, cudaStream_t s) {
  // whole lines per block, about 256 threads, so that the b^2 lines spread over every SM
  const int lpb = b >= 256 ? 1 : 256 / b;
  const int threads = ((lpb * b + 31) / 32) * 32;
  const int blocks = (b * b + lpb - 1) / lpb;
  const int smem = (q ? 2 : 1) * lpb * b * (int)sizeof(T);
  const double np = (double)b * b * b;
  // shared memory stays below the 48 KiB default (b <= 512 lines of at most 2 x 512 values)
  launch_begin(kClassDiv, s);
  if (D.width == 7)
    launch_k(k_div_band_x1<T, 7>, blocks, threads, smem, s, u1, u2, u3, a, b, q, nu, D, lpb, y0, y1);
  else if (D.width == 9)
    launch_k(k_div_band_x1<T, 9>, blocks, threads, smem, s, u1, u2, u3, a, b, q, nu, D, lpb, y0, y1);
  else
    launch_k(k_div_band_x1<T, 0>, blocks, threads, smem, s, u1, u2, u3, a, b, q, nu, D, lpb, y0, y1);
  launch_end(kClassDiv, s, (q ? 8.0 : 6.0) * np + (q ? 4.0 : 2.0) * D.width * np,
             (3.0 * a * b * b + (q ? 3.0 : 1.0) * np) * sizeof(T));
}

template <typename T>
void divergence_plus(const T* u1, const T* u2, const T* u3, int a, int b, T* delta, const T* q,
                     T nu, T* e, cudaStream_t s, int nb, int64_t bs) {
  if (nb < 1) nb = 1;
  const int64_t total = (int64_t)b * b * b * nb;
  launch_begin(kClassDiv, s);
  launch_k(k_divergence<T>, grid_for((int64_t)b * b * nb * 32, 256), 256, 0, s, u1, u2, u3, a, b,
           delta, q, nu, e, nb, bs);
  launch_end(kClassDiv, s, 8.0 * total, (3.0 * a * b * b * nb + 3.0 * total) * sizeof(T));
}

template <typename T>
void div_transpose(const T* g, int a, int b, T* y1, T* y2, T* y3, int accumulate,
                   cudaStream_t s, int nb, int64_t bs) {
  if (nb < 1) nb = 1;
  const int64_t total = 3 * (int64_t)a * b * b * nb;
  launch_begin(kClassDiv, s);
  launch_k(k_div_transpose<T>, grid_for((int64_t)(b * b + 2 * a * b) * nb * 32, 256), 256, 0, s, g,
           a, b, y1, y2, y3, accumulate, nb, bs);
  launch_end(kClassDiv, s, (accumulate ? 2.0 : 1.0) * total,
             ((double)b * b * b * nb + (accumulate ? 2.0 : 1.0) * total) * sizeof(T));
}

__global__ void __launch_bounds__(256) k_quad_stress(double* __restrict__ G, double* __restrict__ P,
                                                     const double* __restrict__ w, int nq,
                                                     double nu) {
  pdl_begin();
  const int64_t n3 = (int64_t)nq * nq * nq;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n3;
       o += (int64_t)gridDim.x * blockDim.x) {
    int i1, i2, i3;
    if (n3 < ((int64_t)1 << 31)) {   // 32-bit division (64-bit division runs on the FP64 pipe)
      const int oi = (int)o, q12 = oi / nq;
      i1 = oi - q12 * nq;
      i3 = q12 / nq;
      i2 = q12 - i3 * nq;
    } else {
      const int64_t q12 = o / nq;
      i1 = (int)(o - q12 * nq);
      i3 = (int)(q12 / nq);
      i2 = (int)(q12 - (int64_t)i3 * nq);
    }
    const double W = w[i1] * w[i2] * w[i3];
    double g[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) g[k] = G[k * n3 + o];
    const double q = P[o];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        double t = W * (nu * (g[3 * c + d] + g[3 * d + c]));
        if (c == d) t += W * q;
        G[(3 * c + d) * n3 + o] = t;
      }
    P[o] = W * (g[0] + g[4] + g[8]);
  }
}

void quad_stress(double* G, double* P, const double* w, int nq, double nu, cudaStream_t s) {
  const int64_t n3 = (int64_t)nq * nq * nq;
  launch_begin(kClassDiv, s);
  launch_k(k_quad_stress, grid_for(n3, 256), 256, 0, s, G, P, w, nq, nu);
  launch_end(kClassDiv, s, 40.0 * n3, 20.0 * n3 * sizeof(double));
}

template void div_band_x1<double>(const double*, const double*, const double*, int, int,
                                  const double*, double, const BandD<double>&, double*, double*,
                                  cudaStream_t);
template void band_pass<double>(const PassArgs<double>&, cudaStream_t);
template void band_pass<float>(const PassArgs<float>&, cudaStream_t);
template void band_pass_multi<double>(const PassArgs<double>*, int, cudaStream_t);
template void band_pass_multi<float>(const PassArgs<float>*, int, cudaStream_t);
template void divergence<double>(const double*, const double*, const double*, int, int, double*,
                                 cudaStream_t, int, int64_t);
template void divergence<float>(const float*, const float*, const float*, int, int, float*,
                                cudaStream_t, int, int64_t);
template void divergence_plus<double>(const double*, const double*, const double*, int, int,
                                      double*, const double*, double, double*, cudaStream_t, int,
                                      int64_t);
template void divergence_plus<float>(const float*, const float*, const float*, int, int, float*,
                                     const float*, float, float*, cudaStream_t, int, int64_t);
template void div_transpose<double>(const double*, int, int, double*, double*, double*, int,
                                    cudaStream_t, int, int64_t);
template void div_transpose<float>(const float*, int, int, float*, float*, float*, int,
                                   cudaStream_t, int, int64_t);

}  // namespace shp
