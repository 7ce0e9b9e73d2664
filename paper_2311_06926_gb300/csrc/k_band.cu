// Banded Kronecker passes (sum factorisation of App. A.2 with banded 1D factors, Sec. 3.3) and
// the exact discrete divergence / its transpose (App. B.2).
//
// One pass multiplies a 3D tensor along one parametric direction by a banded 1D matrix: each
// output entry is a short dot product of the band row with the input line, read through the
// read-only cache. A pass may sum two such products and add an extra tensor and a difference
// term, so that a whole Kronecker sum is evaluated in few passes.
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

template <typename T, int AXIS>
__global__ void __launch_bounds__(256) k_band_pass(PassArgs<T> a) {
  const Dims out = a.in.with(AXIS, a.D0.rows);
  const int64_t total = out.size();
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total; o += step) {
    const int i1 = (int)(o % out.n1);
    const int64_t t = o / out.n1;
    const int i2 = (int)(t % out.n2);
    const int i3 = (int)(t / out.n2);
    const int i = AXIS == 1 ? i1 : (AXIS == 2 ? i2 : i3);
    int64_t base, stride;
    if (AXIS == 1) {
      base = (int64_t)a.in.n1 * (i2 + (int64_t)a.in.n2 * i3);
      stride = 1;
    } else if (AXIS == 2) {
      base = i1 + (int64_t)a.in.n1 * a.in.n2 * i3;
      stride = a.in.n1;
    } else {
      base = i1 + (int64_t)a.in.n1 * i2;
      stride = (int64_t)a.in.n1 * a.in.n2;
    }
    T acc = 0;
    {
      const int s0 = __ldg(a.D0.start + i);
      const T* v = a.D0.val + (int64_t)i * a.D0.width;
      const T* x = a.X0 + base + (int64_t)s0 * stride;
      T s = 0;
      for (int w = 0; w < a.D0.width; ++w) s += __ldg(v + w) * __ldg(x + (int64_t)w * stride);
      acc = a.c0 * s;
    }
    if (a.nterms > 1) {
      const int s1 = __ldg(a.D1.start + i);
      const T* v = a.D1.val + (int64_t)i * a.D1.width;
      const T* x = a.X1 + base + (int64_t)s1 * stride;
      T s = 0;
      for (int w = 0; w < a.D1.width; ++w) s += __ldg(v + w) * __ldg(x + (int64_t)w * stride);
      acc += a.c1 * s;
    }
    if (a.Z) acc += a.cz * a.Z[o];
    if (a.g) {
      // (D^T g) along gaxis: g_j - g_{j+1}; the other two indices are shared with the output
      const int64_t gi = i1 + (int64_t)a.gdims.n1 * (i2 + (int64_t)a.gdims.n2 * i3);
      const int64_t gs = a.gaxis == 1 ? 1 : (a.gaxis == 2 ? (int64_t)a.gdims.n1
                                                         : (int64_t)a.gdims.n1 * a.gdims.n2);
      acc += a.g[gi] - a.g[gi + gs];
    }
    a.Y[o] = acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_divergence(const T* __restrict__ u1, const T* __restrict__ u2,
                                                    const T* __restrict__ u3, int a, int b,
                                                    T* __restrict__ delta) {
  const int64_t total = (int64_t)b * b * b;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total; o += step) {
    const int i1 = (int)(o % b);
    const int i2 = (int)((o / b) % b);
    const int i3 = (int)(o / ((int64_t)b * b));
    T d = 0;
    // u1 extents (a, b, b)
    {
      const int64_t row = (int64_t)a * (i2 + (int64_t)b * i3);
      if (i1 < a) d += u1[row + i1];
      if (i1 >= 1) d -= u1[row + i1 - 1];
    }
    // u2 extents (b, a, b)
    {
      const int64_t off = i1 + (int64_t)b * a * i3;
      if (i2 < a) d += u2[off + (int64_t)b * i2];
      if (i2 >= 1) d -= u2[off + (int64_t)b * (i2 - 1)];
    }
    // u3 extents (b, b, a)
    {
      const int64_t off = i1 + (int64_t)b * i2;
      if (i3 < a) d += u3[off + (int64_t)b * b * i3];
      if (i3 >= 1) d -= u3[off + (int64_t)b * b * (i3 - 1)];
    }
    delta[o] = d;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_div_transpose(const T* __restrict__ g, int a, int b, T* y1,
                                                       T* y2, T* y3, int accumulate) {
  const int64_t nc = (int64_t)a * b * b;
  const int64_t total = 3 * nc;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total; o += step) {
    const int c = (int)(o / nc);
    const int64_t r = o - c * nc;
    T* y = c == 0 ? y1 : (c == 1 ? y2 : y3);
    int i1, i2, i3;
    int64_t gs;
    if (c == 0) {
      i1 = (int)(r % a); i2 = (int)((r / a) % b); i3 = (int)(r / ((int64_t)a * b)); gs = 1;
    } else if (c == 1) {
      i1 = (int)(r % b); i2 = (int)((r / b) % a); i3 = (int)(r / ((int64_t)a * b)); gs = b;
    } else {
      i1 = (int)(r % b); i2 = (int)((r / b) % b); i3 = (int)(r / ((int64_t)b * b));
      gs = (int64_t)b * b;
    }
    const int64_t gi = i1 + (int64_t)b * (i2 + (int64_t)b * i3);
    const T v = g[gi] - g[gi + gs];
    y[r] = accumulate ? y[r] + v : v;
  }
}

}  // namespace

template <typename T>
void band_pass(const PassArgs<T>& a, cudaStream_t s) {
  const Dims out = a.in.with(a.axis, a.D0.rows);
  const int threads = 256;
  const int grid = grid_for(out.size(), threads);
  // algorithmic work: one band row per output and term; one read of every input tensor
  const double outs = (double)out.size();
  double flops = 2.0 * a.D0.width * outs, bytes = (double)a.in.size() + outs;
  if (a.nterms > 1) { flops += 2.0 * a.D1.width * outs; bytes += (double)a.in.size(); }
  if (a.Z) { flops += 2.0 * outs; bytes += outs; }
  if (a.g) { flops += 2.0 * outs; bytes += (double)a.gdims.size(); }
  launch_begin(kClassBand, s);
  if (a.axis == 1) k_band_pass<T, 1><<<grid, threads, 0, s>>>(a);
  else if (a.axis == 2) k_band_pass<T, 2><<<grid, threads, 0, s>>>(a);
  else k_band_pass<T, 3><<<grid, threads, 0, s>>>(a);
  launch_end(kClassBand, s, flops, bytes * sizeof(T));
}

template <typename T>
void divergence(const T* u1, const T* u2, const T* u3, int a, int b, T* delta, cudaStream_t s) {
  const int64_t total = (int64_t)b * b * b;
  launch_begin(kClassDiv, s);
  k_divergence<T><<<grid_for(total, 256), 256, 0, s>>>(u1, u2, u3, a, b, delta);
  launch_end(kClassDiv, s, 6.0 * total, (3.0 * a * b * b + total) * sizeof(T));
}

template <typename T>
void div_transpose(const T* g, int a, int b, T* y1, T* y2, T* y3, int accumulate,
                   cudaStream_t s) {
  const int64_t total = 3 * (int64_t)a * b * b;
  launch_begin(kClassDiv, s);
  k_div_transpose<T><<<grid_for(total, 256), 256, 0, s>>>(g, a, b, y1, y2, y3, accumulate);
  launch_end(kClassDiv, s, (accumulate ? 2.0 : 1.0) * total,
             ((double)b * b * b + (accumulate ? 2.0 : 1.0) * total) * sizeof(T));
}

template void band_pass<double>(const PassArgs<double>&, cudaStream_t);
template void band_pass<float>(const PassArgs<float>&, cudaStream_t);
template void divergence<double>(const double*, const double*, const double*, int, int, double*,
                                 cudaStream_t);
template void divergence<float>(const float*, const float*, const float*, int, int, float*,
                                cudaStream_t);
template void div_transpose<double>(const double*, int, int, double*, double*, double*, int,
                                    cudaStream_t);
template void div_transpose<float>(const float*, int, int, float*, float*, float*, int,
                                   cudaStream_t);

}  // namespace shp
