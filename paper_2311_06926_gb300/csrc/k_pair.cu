// The saddle-point operator K (Sec. 3.3, Eq. 3.3) in pair-of-FP32 arithmetic, for the Arnoldi
// products w = K z of flexible GMRES when the preconditioner runs in reduced precision.
//
// On this part the FP64 pipe runs at about 1/64 of the FP32 rate, and the FP64 banded passes of
// K are bound by it. Here a value is the unevaluated sum hi + lo of two floats (Dekker, "A
// floating-point technique for extending the available precision", 1971): a product is formed
// exactly as p + e with p = a b rounded and e = fma(a, b, -p), a sum exactly as s + t by Knuth's
// TwoSum, and the rounding errors are carried in the low word. Each multiply-add of a band row
// costs about a dozen FP32 operations instead of one FP64 fused multiply-add, several times
// faster on this part, with about 48 significant bits instead of 53.
//
// The input z of the Arnoldi product is the FP32 output of the preconditioner, so it enters as
// pairs with lo = 0; the result is rounded to FP64. The sequence of passes is that of the FP64
// operator (App. B.2 grad-div factorisation, sum factorisation of the Kronecker products):
//   pair_div_x1:  delta = D_div u, e = nu delta + q, and the M-check pass along x1 of both;
//   pair passes:  the velocity passes along the own direction (K, M), then the first and second
//                 other directions, the pressure-mass passes along x2 and x3 riding with them,
//                 and the D_div^T term of the grad-div part in the last velocity pass.
// The band coefficients (already multiplied by nu, 2 nu where the operator has them) are FP64
// values split into pairs on the host.
#include <algorithm>
#include <atomic>

#include "internal.h"
#include "profile.h"

namespace shp {
namespace {

// s + t == a + b exactly (Knuth's TwoSum; round to nearest, no overflow). The _rn intrinsics
// keep the compiler from contracting or reassociating these operations.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}

__device__ __forceinline__ float2 renorm(float h, float l) {
  float s, t;
  two_sum(h, l, s, t);
  return make_float2(s, t);
}

// (sh, sl) += c x with c a pair and x a float (lo = 0): the exact product c.hi x = p + e, the
// term c.lo x folded into e, p added to sh by TwoSum and every error into sl
__device__ __forceinline__ void mac1(float& sh, float& sl, float2 c, float x) {
  const float p = __fmul_rn(c.x, x);
  float e = __fmaf_rn(c.x, x, -p);
  e = __fmaf_rn(c.y, x, e);
  float s, t;
  two_sum(sh, p, s, t);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(t, e));
}

// (sh, sl) += c x with c, x pairs (the product lo * lo, below the pair's precision, is dropped)
__device__ __forceinline__ void mac2(float& sh, float& sl, float2 c, float2 x) {
  const float p = __fmul_rn(c.x, x.x);
  float e = __fmaf_rn(c.x, x.x, -p);
  e = __fmaf_rn(c.x, x.y, e);
  e = __fmaf_rn(c.y, x.x, e);
  float s, t;
  two_sum(sh, p, s, t);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(t, e));
}

// a + sign b for pairs
__device__ __forceinline__ float2 add2(float2 a, float2 b, float sign) {
  float s, t;
  two_sum(a.x, sign * b.x, s, t);
  t = __fadd_rn(t, __fadd_rn(a.y, sign * b.y));
  return renorm(s, t);
}

// (sh, sl) += sign x for a float x
__device__ __forceinline__ void acc1(float& sh, float& sl, float x) {
  float s, t;
  two_sum(sh, x, s, t);
  sh = s;
  sl = __fadd_rn(sl, t);
}

// hi + lo of a normalised pair (|lo| <= ulp(hi) / 2) rounded to FP64, built from the bits of the
// two floats with integer operations (this part's FP64 pipe issues at 1/64 of the FP32 rate):
// hi is exact in FP64, its 29 low mantissa bits are zero, and lo is at most 2^28 FP64 units in
// the last place of hi, so the sum is hi's bit pattern plus lo / ulp64(hi) rounded to an integer.
// Pairs outside the normal FP32 range of that construction (hi zero, tiny or huge), and the case
// where lo lowers a power of two hi into the binade below, take the FP64 addition.
__device__ __forceinline__ double to_f64(float2 v) {
  const uint32_t hb = __float_as_uint(v.x);
  const int e = (int)((hb >> 23) & 0xFFu);   // biased FP32 exponent of hi
  const uint32_t mant = hb & 0x7FFFFFu;
  const bool down = mant == 0u && v.y != 0.f && ((__float_as_uint(v.y) ^ hb) >> 31);
  if (e < 60 || e > 200 || down) return __dadd_rn((double)v.x, (double)v.y);
  // FP64 bits of hi: same sign, exponent rebiased by 1023 - 127, mantissa shifted by 29
  const uint64_t bits = ((uint64_t)(hb >> 31) << 63) | ((uint64_t)(e + 896) << 52) |
                        ((uint64_t)mant << 29);
  // lo in units of hi's FP64 last place, 2^(e - 127 - 52): scale by 2^(179 - e), exact
  const float scaled = __fmul_rn(v.y, __uint_as_float((uint32_t)(179 - e + 127) << 23));
  const int64_t k = (int64_t)__float2int_rn(scaled);
  // the magnitude of hi's pattern moves by k units in the direction of lo's sign
  const uint64_t out = (hb >> 31) ? bits - (uint64_t)k : bits + (uint64_t)k;
  return __longlong_as_double((long long)out);
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

constexpr int kLines = 32;          // lines per block (one per lane)
constexpr int kRows = 8;            // consecutive outputs per lane (register window)
constexpr int kPitch = kLines + 1;  // shared pitch of the slabs, in elements
constexpr int kThreads = 256;

struct PairBatch {
  PairPass job[kMaxPairJobs];
  int first_block[kMaxPairJobs + 1];
  int njobs;
};

// Rows of a job's slab: the input extent padded to whole row chunks, plus H zero rows above and
// below, so that row i of the output reads slab rows i .. i + 2H with no clamping.
__host__ __device__ inline int slab_rows(int nin, int m, int H) {
  const int mr = (m + kRows - 1) / kRows * kRows;
  return (nin > mr ? nin : mr) + 2 * H;
}

// line (over all items) -> offset of the line in a tensor of extents d (item k at k * bs), and
// the stride along the band direction. 32-bit index arithmetic within an item (the launcher takes
// items below 2^31 entries and fewer than 2^31 lines in all); 64-bit integer division would run
// through the slow FP64 pipe.
__device__ __forceinline__ int64_t line_base(int axis, const Dims& d, int lines1, int64_t bs,
                                             int line, int* stride) {
  const int k = line / lines1, li = line - k * lines1;
  int base;
  if (axis == 1) {
    base = d.n1 * li;
    *stride = 1;
  } else if (axis == 2) {
    const int i3 = li / d.n1, i1 = li - i3 * d.n1;
    base = i1 + d.n1 * d.n2 * i3;
    *stride = d.n1;
  } else {
    base = li;
    *stride = d.n1 * d.n2;
  }
  return (int64_t)k * bs + base;
}

template <int H, typename XT>
__device__ __forceinline__ void chunk_term(const XT* xs, const float2* crow, int pitch,
                                           float (&sh)[kRows], float (&sl)[kRows]) {
  constexpr int W = 2 * H + 1;
  XT v[kRows + 2 * H];
#pragma unroll
  for (int k = 0; k < kRows + 2 * H; ++k) v[k] = xs[k * kPitch];
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    const float4* c4 = reinterpret_cast<const float4*>(crow + r * pitch);
#pragma unroll
    for (int k2 = 0; k2 < (W + 1) / 2; ++k2) {
      const float4 c = __ldg(c4 + k2);
      if constexpr (sizeof(XT) == 4) {
        mac1(sh[r], sl[r], make_float2(c.x, c.y), v[r + 2 * k2]);
        if (2 * k2 + 1 < W) mac1(sh[r], sl[r], make_float2(c.z, c.w), v[r + 2 * k2 + 1]);
      } else {
        mac2(sh[r], sl[r], make_float2(c.x, c.y), v[r + 2 * k2]);
        if (2 * k2 + 1 < W) mac2(sh[r], sl[r], make_float2(c.z, c.w), v[r + 2 * k2 + 1]);
      }
    }
  }
}

// One block: 32 neighbouring lines (lines of all items in memory order) x the whole band extent.
// The input slabs ([row][line], H zero rows above and below) are copied with cp.async, every copy
// in flight before one wait; each lane then forms kRows consecutive outputs of its line from one
// register window of kRows + 2H inputs, the band rows read as float4 (two pairs) through the
// read-only cache. Passes along x1 stage their outputs in shared memory for coalesced stores.
template <int H>
__global__ void __launch_bounds__(kThreads, 2) k_pair_pass(const __grid_constant__ PairBatch pb) {
  pdl_begin();
  extern __shared__ __align__(16) unsigned char pair_smem[];
  int jb = 0;
  while (jb + 1 < pb.njobs && (int)blockIdx.x >= pb.first_block[jb + 1]) ++jb;
  const PairPass& a = pb.job[jb];
  const int axis = a.axis;
  const int nin = a.in.get(axis);
  const int m = a.D[0].rows;
  const int nt = a.nterms;
  const Dims out = a.in.with(axis, m);
  const int lines1 = (int)(out.size() / m);
  const int nb = a.nb > 1 ? a.nb : 1;
  const int lines = lines1 * nb;
  const int line0 = (blockIdx.x - pb.first_block[jb]) * kLines;
  const int nl = lines - line0 < kLines ? lines - line0 : kLines;
  const int rs = slab_rows(nin, m, H);
  const size_t slab_bytes = (size_t)rs * kPitch * 8;
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32, nwarps = kThreads / 32;
  const bool f32 = a.in_f32 != 0;

  for (int t = 0; t < nt; ++t) {
    unsigned char* sb = pair_smem + t * slab_bytes;
    // zero rows: H above, and everything below the input extent
    for (int idx = tid; idx < (rs - nin) * kPitch; idx += kThreads) {
      const int r = idx / kPitch, l = idx - r * kPitch;
      const int row = r < H ? r : nin + r;
      if (f32) reinterpret_cast<float*>(sb)[row * kPitch + l] = 0.f;
      else reinterpret_cast<float2*>(sb)[row * kPitch + l] = make_float2(0.f, 0.f);
    }
    if (axis == 1) {
      for (int l = warp; l < kLines; l += nwarps) {
        int st = 0;
        const int64_t base = l < nl ? line_base(1, a.in, lines1, a.bs, line0 + l, &st) : 0;
        for (int j = lane; j < nin; j += 32) {
          const int o = (j + H) * kPitch + l;
          if (f32) {
            float* d = reinterpret_cast<float*>(sb) + o;
            if (l < nl) cp_async4(d, static_cast<const float*>(a.X[t]) + base + j);
            else *d = 0.f;
          } else {
            float2* d = reinterpret_cast<float2*>(sb) + o;
            if (l < nl) cp_async8(d, static_cast<const float2*>(a.X[t]) + base + j);
            else *d = make_float2(0.f, 0.f);
          }
        }
      }
    } else {
      int st = 0;
      const int64_t base = lane < nl ? line_base(axis, a.in, lines1, a.bs, line0 + lane, &st) : 0;
      for (int j = warp; j < nin; j += nwarps) {
        const int o = (j + H) * kPitch + lane;
        if (f32) {
          float* d = reinterpret_cast<float*>(sb) + o;
          if (lane < nl) cp_async4(d, static_cast<const float*>(a.X[t]) + base + st * j);
          else *d = 0.f;
        } else {
          float2* d = reinterpret_cast<float2*>(sb) + o;
          if (lane < nl) cp_async8(d, static_cast<const float2*>(a.X[t]) + base + st * j);
          else *d = make_float2(0.f, 0.f);
        }
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();

  int64_t obase = 0, gbase = 0;
  int ostride = 0, gstride = 0, gstep = 0;
  if (lane < nl) {
    obase = line_base(axis, out, lines1, a.bs, line0 + lane, &ostride);
    if (a.g) {
      const int line = line0 + lane;
      const int k = line / lines1, li = line - k * lines1;
      // the line's position in the two directions other than the band direction
      int j1 = 0, j2 = 0, j3 = 0;
      if (axis == 1) { j3 = li / out.n2; j2 = li - j3 * out.n2; }
      else if (axis == 2) { j3 = li / out.n1; j1 = li - j3 * out.n1; }
      else { j2 = li / out.n1; j1 = li - j2 * out.n1; }
      const Dims gd = a.gdims;
      const int g2 = gd.n1, g3 = gd.n1 * gd.n2;
      gbase = (int64_t)k * a.bs + (j1 + g2 * j2 + g3 * j3);
      gstride = axis == 1 ? 1 : (axis == 2 ? g2 : g3);
      gstep = a.gaxis == 1 ? 1 : (a.gaxis == 2 ? g2 : g3);
    }
  }
  unsigned char* ys = pair_smem + nt * slab_bytes;   // m x kPitch outputs (passes along x1)
  const int nchunks = (m + kRows - 1) / kRows;
  for (int ch = warp; ch < nchunks; ch += nwarps) {
    const int i0 = ch * kRows;
    float sh[kRows], sl[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) sh[r] = sl[r] = 0.f;
    for (int t = 0; t < nt; ++t) {
      const unsigned char* sb = pair_smem + t * slab_bytes;
      const float2* crow = a.D[t].c + (size_t)i0 * a.D[t].pitch;
      if (f32)
        chunk_term<H>(reinterpret_cast<const float*>(sb) + i0 * kPitch + lane, crow, a.D[t].pitch,
                      sh, sl);
      else
        chunk_term<H>(reinterpret_cast<const float2*>(sb) + i0 * kPitch + lane, crow,
                      a.D[t].pitch, sh, sl);
    }
    if (lane < nl) {
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        const int i = i0 + r;
        if (i >= m) break;
        float2 y = renorm(sh[r], sl[r]);
        if (a.g) {
          const int64_t gi = gbase + gstride * i;
          y = add2(y, add2(a.g[gi], a.g[gi + gstep], -1.f), 1.f);
        }
        if (axis == 1) {
          if (a.out_f64) reinterpret_cast<double*>(ys)[i * kPitch + lane] = to_f64(y);
          else reinterpret_cast<float2*>(ys)[i * kPitch + lane] = y;
        } else {
          const int64_t o = obase + ostride * i;
          if (a.out_f64) static_cast<double*>(a.Y)[o] = to_f64(y);
          else static_cast<float2*>(a.Y)[o] = y;
        }
      }
    }
  }
  if (axis == 1) {
    __syncthreads();
    for (int l = warp; l < nl; l += nwarps) {
      int st = 0;
      const int64_t base = line_base(1, out, lines1, a.bs, line0 + l, &st);
      if (a.out_f64) {
        double* row = static_cast<double*>(a.Y) + base;
        for (int i = lane; i < m; i += 32) row[i] = reinterpret_cast<const double*>(ys)[i * kPitch + l];
      } else {
        float2* row = static_cast<float2*>(a.Y) + base;
        for (int i = lane; i < m; i += 32) row[i] = reinterpret_cast<const float2*>(ys)[i * kPitch + l];
      }
    }
  }
}

// delta = D_div u (App. B.2: (D beta)_i = beta_i - beta_{i-1}, beta_{-1} = beta_a = 0 along each
// component's own direction), e = nu delta + q, both as pairs, and their M-check pass along x1.
// A block owns lpb whole x1 lines of the pressure grid (lines of all items in order); the line
// values go to shared memory with H zero entries on either side, and each thread forms one
// output of both passes.
template <int H>
__global__ void __launch_bounds__(256) k_pair_div_x1(const float* __restrict__ u1,
                                                     const float* __restrict__ u2,
                                                     const float* __restrict__ u3,
                                                     const float* __restrict__ q, int a, int b,
                                                     float2 nu, const __grid_constant__ PairBand D,
                                                     int lpb, float2* __restrict__ y0,
                                                     float2* __restrict__ y1, int nb, int64_t bs) {
  constexpr int W = 2 * H + 1;
  pdl_begin();
  extern __shared__ __align__(16) unsigned char pdiv_smem[];
  const int ld = b + 2 * H;
  float2* sd = reinterpret_cast<float2*>(pdiv_smem);   // [lpb][ld]: delta
  float2* se = sd + lpb * ld;                          // [lpb][ld]: e
  const int lines1 = b * b;
  const int t = threadIdx.x;
  const int l = t / b, i1 = t - l * b;
  const int line = blockIdx.x * lpb + l;
  const bool active = l < lpb && line < lines1 * nb;
  for (int idx = t; idx < lpb * 2 * H; idx += blockDim.x) {
    const int ll = idx / (2 * H), r = idx - ll * (2 * H);
    const int col = r < H ? r : b + r;
    sd[ll * ld + col] = make_float2(0.f, 0.f);
    se[ll * ld + col] = make_float2(0.f, 0.f);
  }
  int64_t kb = 0;
  int li = 0;
  if (active) {
    const int k = line / lines1;
    kb = (int64_t)k * bs;
    li = line - k * lines1;
    const int i3 = li / b, i2 = li - i3 * b;
    const float* v1 = u1 + kb;
    const float* v2 = u2 + kb;
    const float* v3 = u3 + kb;
    float dh = 0.f, dl = 0.f;
    {
      const int row = a * (i2 + b * i3);
      if (i1 < a) acc1(dh, dl, v1[row + i1]);
      if (i1 >= 1) acc1(dh, dl, -v1[row + i1 - 1]);
    }
    {
      const int off = i1 + b * a * i3;
      if (i2 < a) acc1(dh, dl, v2[off + b * i2]);
      if (i2 >= 1) acc1(dh, dl, -v2[off + b * (i2 - 1)]);
    }
    {
      const int off = i1 + b * i2;
      if (i3 < a) acc1(dh, dl, v3[off + b * b * i3]);
      if (i3 >= 1) acc1(dh, dl, -v3[off + b * b * (i3 - 1)]);
    }
    const float2 d = renorm(dh, dl);
    // e = nu delta + q: the exact product nu.hi d.hi, its error and the cross terms, then q
    float ph = __fmul_rn(nu.x, d.x);
    float pl = __fmaf_rn(nu.x, d.x, -ph);
    pl = __fmaf_rn(nu.x, d.y, pl);
    pl = __fmaf_rn(nu.y, d.x, pl);
    acc1(ph, pl, q[kb + (li * b + i1)]);
    sd[l * ld + H + i1] = d;
    se[l * ld + H + i1] = renorm(ph, pl);
  }
  __syncthreads();
  if (!active) return;
  const float2* cr = D.c + (size_t)i1 * D.pitch;
  const float2* xd = sd + l * ld + i1;
  const float2* xe = se + l * ld + i1;
  float dh = 0.f, dl = 0.f, eh = 0.f, el = 0.f;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const float2 c = __ldg(cr + k);
    mac2(dh, dl, c, xd[k]);
    mac2(eh, el, c, xe[k]);
  }
  const int64_t o = kb + (li * b + i1);
  y0[o] = renorm(dh, dl);
  y1[o] = renorm(eh, el);
}

}  // namespace

cudaError_t pair_pass_multi(const PairPass* jobs, int njobs, int H, cudaStream_t s) {
  if (njobs < 1 || njobs > kMaxPairJobs || H < 1 || H > 6) return cudaErrorInvalidValue;
  // 32-bit index arithmetic within an item and over the lines of all items
  for (int j = 0; j < njobs; ++j) {
    const PairPass& a = jobs[j];
    const Dims out = a.in.with(a.axis, a.D[0].rows);
    const int64_t lines = out.size() / a.D[0].rows * std::max(a.nb, 1);
    if (std::max(a.in.size(), out.size()) >= ((int64_t)1 << 31) || lines + kLines >= ((int64_t)1 << 31))
      return cudaErrorInvalidValue;
  }
  PairBatch pb{};
  pb.njobs = njobs;
  int blocks = 0;
  size_t smem = 0;
  double flops = 0, bytes = 0;
  for (int j = 0; j < njobs; ++j) {
    const PairPass& a = jobs[j];
    pb.job[j] = a;
    pb.first_block[j] = blocks;
    const int m = a.D[0].rows;
    const Dims out = a.in.with(a.axis, m);
    const int nbj = a.nb > 1 ? a.nb : 1;
    const int64_t lines = out.size() / m * nbj;
    blocks += (int)((lines + kLines - 1) / kLines);
    const size_t sm = (size_t)a.nterms * slab_rows(a.in.get(a.axis), m, H) * kPitch * 8 +
                      (a.axis == 1 ? (size_t)m * kPitch * 8 : 0);
    smem = std::max(smem, sm);
    // algorithmic work: one band row of 2H + 1 entries per output and term (multiply-adds as
    // 2 flops each), one read of every input tensor, one write of the output
    const double outs = (double)out.size() * nbj;
    flops += 2.0 * (2 * H + 1) * outs * a.nterms;
    bytes += a.nterms * (double)a.in.size() * nbj * (a.in_f32 ? 4.0 : 8.0) + outs * 8.0;
    if (a.g) bytes += (double)a.gdims.size() * nbj * 8.0;
  }
  pb.first_block[njobs] = blocks;
  cudaError_t err = cudaSuccess;
  launch_begin(kClassPair, s);
  switch (H) {
#define SHP_PAIR_H(h)                                                          \
  case h: {                                                                    \
    static std::atomic<int> attr{0};                                           \
    err = raise_smem_limit(k_pair_pass<h>, attr, (int)smem);                   \
    if (err == cudaSuccess) err = launch_k(k_pair_pass<h>, blocks, kThreads, (int)smem, s, pb); \
    break;                                                                     \
  }
    SHP_PAIR_H(1) SHP_PAIR_H(2) SHP_PAIR_H(3) SHP_PAIR_H(4) SHP_PAIR_H(5) SHP_PAIR_H(6)
#undef SHP_PAIR_H
  }
  launch_end(kClassPair, s, flops, bytes);
  return err;
}

cudaError_t pair_div_x1(const float* u1, const float* u2, const float* u3, const float* q, int a,
                        int b, float2 nu, const PairBand& D, int H, float2* y0, float2* y1,
                        int nb, int64_t bs, cudaStream_t s) {
  if (H < 1 || H > 6 || b < 1 || b > 256) return cudaErrorInvalidValue;
  if (nb < 1) nb = 1;
  if ((int64_t)b * b * nb >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
  const int lpb = std::max(1, 256 / b);
  const int threads = ((lpb * b + 31) / 32) * 32;
  const int64_t lines = (int64_t)b * b * nb;
  const int blocks = (int)((lines + lpb - 1) / lpb);
  const int smem = 2 * lpb * (b + 2 * H) * (int)sizeof(float2);
  const double np = (double)b * b * b * nb;
  cudaError_t err = cudaSuccess;
  launch_begin(kClassPair, s);
  switch (H) {
#define SHP_PDIV_H(h)                                                                          \
  case h: {                                                                                    \
    static std::atomic<int> attr{0};                                                           \
    err = raise_smem_limit(k_pair_div_x1<h>, attr, smem);                                      \
    if (err == cudaSuccess)                                                                    \
      err = launch_k(k_pair_div_x1<h>, blocks, threads, smem, s, u1, u2, u3, q, a, b, nu, D,   \
                     lpb, y0, y1, nb, bs);                                                     \
    break;                                                                                     \
  }
    SHP_PDIV_H(1) SHP_PDIV_H(2) SHP_PDIV_H(3) SHP_PDIV_H(4) SHP_PDIV_H(5) SHP_PDIV_H(6)
#undef SHP_PDIV_H
  }
  launch_end(kClassPair, s, 8.0 * np + 4.0 * (2 * H + 1) * np,
             (3.0 * a * b * b * nb + np) * 4.0 + 2.0 * np * 8.0);
  return err;
}

}  // namespace shp
