// Context, operator sequences, hyper-power recursion, Krylov drivers and the C ABI.
//
// Operators (Sec. 3.3). Because interior N-splines vanish at both ends of [0, 1], integration by
// parts and the derivative identity of App. B.2 give C = -D^T M-check and C-check = D^T M-check,
// with D the (b x a) coefficient difference (D beta)_i = beta_i - beta_{i-1}. The six printed
// off-diagonal Kronecker products of A and the three of B then factor through the pressure mass
// matrix M_q = M-check^3 and the exact discrete divergence D_div:
//   B = D_div^T M_q,   B^T = M_q D_div,
//   A = blockdiag(A'_cc) + nu D_div^T M_q D_div,   A'_cc = A_cc - nu D_c^T M_q D_c,
// where D_c^T M_q D_c = (mass) (x) (mass) (x) K in direction c because K = D^T M-check D. For
// component 1, A'_11 = nu Mc (x) Mc (x) K + 2 nu (Mc (x) Tc (x) M + Tc (x) Mc (x) M). This is
// the same matrix as the 15 printed products, evaluated with fewer banded passes.
//
// Base preconditioner (Eq. 4.1): fast diagonalisation of the diagonal blocks A_cc (App. A.4) and
// the pressure block M_q / (2 nu), whose inverse 2 nu (U_T U_T^T)^(x)3 reuses the (T-check,
// M-check) eigenvectors: U_T^T M-check U_T = I gives M-check^-1 = U_T U_T^T.
//
// Hyper-power sequence of order q (Eq. 2.1 for q = 2): X_{k+1} x = X_k sum_{j<q} (I - A~ X_k)^j x,
// evaluated as r = x, acc = x, then (q - 1) times {r -= A~ X_k r; acc += r}, then X_k acc.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <type_traits>
#include <utility>
#include <vector>

#include "host_setup.h"
#include "internal.h"
#include "mma.h"
#include "profile.h"
#include "stokes_hp.h"

namespace shp {
namespace {

struct CudaError {
  cudaError_t e;
  const char* what;
};

inline void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw CudaError{e, what};
}

struct ArgError {
  std::string msg;
};
struct SetupError {
  std::string msg;
};

// ---- device memory owned by a context ---------------------------------------------------------
struct Arena {
  std::vector<void*> ptrs;
  template <typename T>
  T* alloc(size_t count) {
    void* p = nullptr;
    if (count == 0) count = 1;
    ck(cudaMalloc(&p, count * sizeof(T)), "cudaMalloc");
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  ~Arena() {
    for (void* p : ptrs) cudaFree(p);
  }
};

// The same banded matrix stored with a larger band width (zeros in the added slots); rows = 0 when
// the matrix has fewer columns than the width.
// s B (entrywise, FP64)
Band scaled(const Band& B, double sc) {
  Band S = B;
  for (double& v : S.val) v *= sc;
  return S;
}

Band widen(const Band& B, int width) {
  Band W;
  if (width <= B.width || B.cols < width) return W;
  const int d = (width - B.width) / 2;
  W.rows = B.rows;
  W.cols = B.cols;
  W.width = width;
  W.start.resize(B.rows);
  W.val.assign((size_t)B.rows * width, 0.0);
  for (int i = 0; i < B.rows; ++i) {
    const int s0 = std::max(0, std::min(B.start[i] - d, B.cols - width));
    W.start[i] = s0;
    for (int w = 0; w < B.width; ++w)
      W.val[(size_t)i * width + (B.start[i] + w - s0)] = B.val[(size_t)i * B.width + w];
  }
  return W;
}

// min_half: lower bound of the centred copy's half width (a zero-padded copy keeps the width of
// the matrices it shares launches with)
template <typename T>
BandD<T> upload_band(Arena& ar, const Band& b, cudaStream_t s, int min_half = 0) {
  BandD<T> d;
  d.rows = b.rows;
  d.cols = b.cols;
  d.width = b.width;
  int* st = ar.alloc<int>(b.start.size());
  T* v = ar.alloc<T>(b.val.size());
  std::vector<T> tv(b.val.begin(), b.val.end());
  ck(cudaMemcpyAsync(st, b.start.data(), b.start.size() * sizeof(int), cudaMemcpyHostToDevice, s),
     "upload band");
  ck(cudaMemcpyAsync(v, tv.data(), tv.size() * sizeof(T), cudaMemcpyHostToDevice, s),
     "upload band");
  d.start = st;
  d.val = v;
  {
    // transposed copy for the passes along x1 whose lanes take consecutive rows
    std::vector<T> tt((size_t)b.rows * b.width);
    for (int i = 0; i < b.rows; ++i)
      for (int w = 0; w < b.width; ++w)
        tt[(size_t)w * b.rows + i] = (T)b.val[(size_t)i * b.width + w];
    T* vt = ar.alloc<T>(tt.size());
    ck(cudaMemcpyAsync(vt, tt.data(), tt.size() * sizeof(T), cudaMemcpyHostToDevice, s),
       "upload band");
    d.valT = vt;
  }
  d.cval = nullptr;
  d.half = 0;
  d.cpitch = 0;
  d.tlo = d.thi = 0;
  // centred copy for square matrices (every matrix of the operator applies is one)
  std::vector<T> cv;
  if (b.rows == b.cols) {
    int half = min_half;
    for (int i = 0; i < b.rows; ++i)
      for (int w = 0; w < b.width; ++w)
        if (b.val[(size_t)i * b.width + w] != 0.0) half = std::max(half, std::abs(b.start[i] + w - i));
    const int pitch = (2 * half + 4) & ~3;
    const int rows8 = (b.rows + 7) / 8 * 8;
    cv.assign((size_t)rows8 * pitch, T(0));
    for (int i = 0; i < b.rows; ++i)
      for (int w = 0; w < b.width; ++w) {
        const int k = b.start[i] + w - i + half;
        if (k >= 0 && k <= 2 * half && b.start[i] + w < b.cols)
          cv[(size_t)i * pitch + k] = (T)b.val[(size_t)i * b.width + w];
      }
    // Toeplitz interior: rows equal to the middle row. In FP32 an interior entry may round to a
    // neighbouring float of the middle row's (the FP64 entries agree to rounding only); entries
    // within 2 float ulps of the middle row's are set to it, so one coefficient set serves every
    // interior row.
    d.tlo = d.thi = 0;
    if (sizeof(T) == 4 && b.rows >= 8) {
      const int mid = b.rows / 2;
      auto same = [&](int i) {
        for (int k = 0; k < pitch; ++k) {
          const double x = (double)cv[(size_t)i * pitch + k], y = (double)cv[(size_t)mid * pitch + k];
          if (std::fabs(x - y) > 2.0 * 1.1920928955078125e-07 * std::fabs(y)) return false;
        }
        return true;
      };
      int lo = mid, hi = mid + 1;
      while (lo > 0 && same(lo - 1)) --lo;
      while (hi < b.rows && same(hi)) ++hi;
      for (int i = lo; i < hi; ++i)
        for (int k = 0; k < pitch; ++k) cv[(size_t)i * pitch + k] = cv[(size_t)mid * pitch + k];
      d.tlo = lo;
      d.thi = hi;
    }
    T* c = ar.alloc<T>(cv.size());
    ck(cudaMemcpyAsync(c, cv.data(), cv.size() * sizeof(T), cudaMemcpyHostToDevice, s),
       "upload band");
    d.cval = c;
    d.half = half;
    d.cpitch = pitch;
  }
  ck(cudaStreamSynchronize(s), "upload band");
  return d;
}

template <typename T>
T* upload(Arena& ar, const std::vector<double>& h, cudaStream_t s) {
  T* d = ar.alloc<T>(h.size());
  std::vector<T> tv(h.begin(), h.end());
  ck(cudaMemcpyAsync(d, tv.data(), tv.size() * sizeof(T), cudaMemcpyHostToDevice, s), "upload");
  ck(cudaStreamSynchronize(s), "upload");
  return d;
}

// One hyper-power Horner step applied by the pass that produces A~ t (see PassArgs): mode 1 sets
// r = x - A~ t, acc = x + r; mode 2 sets r = r - A~ t, acc = acc + r. r, acc, x have the layout of
// the product.
template <typename T>
struct Horner {
  int mode;
  T* r;
  T* acc;
  const T* x;
};

// ---- operators in precision T ------------------------------------------------------------------
template <typename T>
struct Ops {
  int a = 0, b = 0;
  T nu = 0;
  int64_t nvc = 0, nvel = 0, npres = 0;
  BandD<T> M{}, K{}, Mc{}, Tc{};
  BandD<T> Mc_w{};   // M-check padded with zeros to the band width of K and M (val null: none)
  // FP64: nu M-check and 2 nu T-check, so that the two terms of a velocity pass form one FMA
  // chain with unit coefficients (each product by nu, 2 nu is one FP64 instruction fewer per
  // output on the FP64-bound passes)
  BandD<T> Mc_nu{}, Tc_2nu{};
  const T *U_N = nullptr, *lam_N = nullptr, *U_T = nullptr, *lam_T = nullptr;
  const T* invd = nullptr;   // FP64: 1 / (2 nu (l1 + l2 + l3)) per velocity entry
  int eo_N = 0, eo_T = 0;    // FP64: even-mode counts of the parity-split eigenvectors
  int fd_fused = 0;          // FP64: fast diagonalisation by the fused plane / x3-line kernels,
                             // with this many blocks per plane (0: six single-direction passes)
  const T* chol_lb = nullptr;          // pressure block: banded Cholesky factor of M-check
  const T* chol_inv = nullptr;
  int chol_p = 0;
  T *tK = nullptr, *tM = nullptr, *tS = nullptr, *tR = nullptr;   // component-size temporaries
  T *f1 = nullptr, *f2 = nullptr;                                 // mode-product ping-pong
  T *delta = nullptr, *m1 = nullptr, *m2 = nullptr;               // pressure-size temporaries
  cudaStream_t s = nullptr;
  // batch: nb items per vector, item k of every tensor bs elements after item k - 1's
  int nb = 1;
  int64_t bs = 0;
  // FP64 launch shapes (threads per block) chosen by the setup tuner
  int mode_block = 512, band_block = 256;
  // tensor-core fast diagonalisation (reduced precision only): per tensor (3 velocity components,
  // pressure) a padded input copy and six rotating mode products
  bool tc = false;
  bool tc_bf16 = false;
  int sms = 152;
  int* tc_err = nullptr;
  uint32_t tc_spin = 0;         // polls per pipeline wait of the tensor-core kernel (0: default)
  int tc_nsplit = 1;            // tensor-core tile shape: N columns of a tile in 1 or 2 work units
  void* tc_p0[4] = {nullptr, nullptr, nullptr, nullptr};
  int tc_ld0[4] = {0, 0, 0, 0};
  RmpPlan* tc_plan = nullptr;   // [4][6], host memory

  Dims comp(int c) const {
    if (c == 0) return Dims{a, b, b};
    if (c == 1) return Dims{b, a, b};
    return Dims{b, b, a};
  }

  PassArgs<T> job(const T* X0, const BandD<T>& D0, T c0, const T* X1, const BandD<T>* D1, T c1,
                  Dims in, int axis, T* Y, const T* Z = nullptr, T cz = 0, const T* g = nullptr,
                  int gaxis = 0) const {
    PassArgs<T> p{};
    p.X0 = X0;
    p.D0 = D0;
    p.c0 = c0;
    p.X1 = X1;
    p.D1 = D1 ? *D1 : D0;
    p.c1 = c1;
    p.nterms = X1 ? 2 : 1;
    p.Z = Z;
    p.cz = cz;
    p.g = g;
    p.gaxis = gaxis;
    p.gdims = Dims{b, b, b};
    p.Y = Y;
    p.in = in;
    p.axis = axis;
    p.nb = nb;
    p.bs = bs;
    p.block = band_block;
    return p;
  }

  // the job's result goes through the Horner epilogue h (offset o into its vectors)
  static void horner(PassArgs<T>& p, const Horner<T>* h, int64_t o) {
    if (!h) return;
    p.hmode = h->mode;
    p.hr = h->r + o;
    p.hacc = h->acc + o;
    p.hx = h->x ? h->x + o : nullptr;
  }

  static int own_axis(int c) { return c + 1; }
  static int first_other(int c) { return c == 0 ? 2 : 1; }
  static int second_other(int c) { return c == 2 ? 2 : 3; }

  // y_c = A'_cc u_c + D^T g along the own direction of c, for the three components at once:
  // t_K = K u, t_M = M u along the own direction; s = nu Mc t_K + 2 nu Tc t_M and r = Mc t_M
  // along the first other direction; y = Mc s + 2 nu Tc r (+ D^T g) along the second.
  // With nq > 0 the pressure-mass products g_k = coef_k M_q x_k (k < nq) that feed g are formed in
  // the same launches: their passes along x1 and x2 ride with the first two velocity passes (the
  // x1 pass with Mc_w, M-check padded with zeros to the width of K and M, so that every job of a
  // launch has one band width), their pass along x3 runs alone, then the last velocity pass.
  // x1_done: the inputs qx already carry the pass along x1 (div_band_x1); their passes along x2
  // (with Mc_w) and x3 then ride with the first and second velocity passes, and no pressure-mass
  // launch of its own remains.
  void adiag_all(const T* u, T* y, const T* g, int nq = 0, const T* const* qx = nullptr,
                 T* const* qy = nullptr, const T* qcoef = nullptr,
                 const Horner<T>* h = nullptr, bool x1_done = false) const {
    const T nu2 = 2 * nu;
    const Dims dq{b, b, b};
    PassArgs<T> j[kMaxPassJobs];
    for (int c = 0; c < 3; ++c) {
      const int64_t o = c * nvc;
      j[2 * c] = job(u + o, K, 1, nullptr, nullptr, 0, comp(c), own_axis(c), tK + o);
      j[2 * c + 1] = job(u + o, M, 1, nullptr, nullptr, 0, comp(c), own_axis(c), tM + o);
    }
    // the x2 pass rides with M-check itself (FP64 launches take jobs of width 7 along x2 in a
    // width-9 launch); the x1 pass, where the flat layout needs the launch's width, with the
    // zero-padded copy
    for (int k = 0; k < nq; ++k)
      j[6 + k] = x1_done ? job(qx[k], std::is_same<T, double>::value ? Mc : Mc_w, 1, nullptr,
                               nullptr, 0, dq, 2, f2 + k * npres)
                         : job(qx[k], Mc_w, 1, nullptr, nullptr, 0, dq, 1, f1 + k * npres);
    band_pass_multi<T>(j, 6 + nq, s);
    const bool chain = Mc_nu.val != nullptr;   // FP64: one FMA chain over both terms
    for (int c = 0; c < 3; ++c) {
      const int64_t o = c * nvc;
      j[2 * c] = chain ? job(tK + o, Mc_nu, 1, tM + o, &Tc_2nu, 1, comp(c), first_other(c), tS + o)
                       : job(tK + o, Mc, nu, tM + o, &Tc, nu2, comp(c), first_other(c), tS + o);
      j[2 * c + 1] = job(tM + o, Mc, 1, nullptr, nullptr, 0, comp(c), first_other(c), tR + o);
    }
    for (int k = 0; k < nq; ++k)
      j[6 + k] = x1_done
                     ? job(f2 + k * npres, Mc, qcoef[k], nullptr, nullptr, 0, dq, 3, qy[k])
                     : job(f1 + k * npres, Mc, 1, nullptr, nullptr, 0, dq, 2, f2 + k * npres);
    band_pass_multi<T>(j, 6 + nq, s);
    if (nq > 0 && !x1_done) {
      for (int k = 0; k < nq; ++k)
        j[k] = job(f2 + k * npres, Mc, qcoef[k], nullptr, nullptr, 0, dq, 3, qy[k]);
      band_pass_multi<T>(j, nq, s);
    }
    for (int c = 0; c < 3; ++c) {
      const int64_t o = c * nvc;
      j[c] = chain ? job(tS + o, Mc, 1, tR + o, &Tc_2nu, 1, comp(c), second_other(c), y + o,
                         nullptr, 0, g, own_axis(c))
                   : job(tS + o, Mc, 1, tR + o, &Tc, nu2, comp(c), second_other(c), y + o,
                         nullptr, 0, g, own_axis(c));
      horner(j[c], h, o);
    }
    band_pass_multi<T>(j, 3, s);
  }

  // y_k = coef_k M_q x_k for nvec <= 2 independent vectors (M_q = M-check^(x)3); h: Horner step
  // applied to the (single) result
  // x1_done: the pass along x1 has already been applied, its results are in f1 + k npres.
  void mq(int nvec, const T* const* x, T* const* y, const T* coef,
          const Horner<T>* h = nullptr, bool x1_done = false) const {
    const Dims d{b, b, b};
    PassArgs<T> j[2];
    if (!x1_done) {
      for (int k = 0; k < nvec; ++k)
        j[k] = job(x[k], Mc, 1, nullptr, nullptr, 0, d, 1, f1 + k * npres);
      band_pass_multi<T>(j, nvec, s);
    }
    for (int k = 0; k < nvec; ++k)
      j[k] = job(f1 + k * npres, Mc, 1, nullptr, nullptr, 0, d, 2, f2 + k * npres);
    band_pass_multi<T>(j, nvec, s);
    for (int k = 0; k < nvec; ++k) {
      j[k] = job(f2 + k * npres, Mc, coef[k], nullptr, nullptr, 0, d, 3, y[k]);
      if (nvec == 1) horner(j[k], h, 0);
    }
    band_pass_multi<T>(j, nvec, s);
  }

  // FP64, one item: the divergence and the pressure-mass pass along x1 fused (div_band_x1), so
  // an A or K apply takes four launches
  bool fused_div() const {
    return std::is_same<T, double>::value && nb == 1 && Mc_w.val != nullptr && b <= 512;
  }

  void apply_K(const T* x, T* y) const {
    const T* q = x + nvel;
    T* yq = y + nvel;
    if constexpr (std::is_same<T, double>::value) {
      if (fused_div()) {
        // the x1 pass with M-check itself (width 7): the zero-padded copy Mc_w that the x2 pass
        // rides with (the velocity launch of width 9) would add two FMAs by zero per output
        div_band_x1<T>(x, x + nvc, x + 2 * nvc, a, b, q, nu, Mc, f1, f1 + npres, s);
        const T* in2[2] = {f1, f1 + npres};
        T* out2[2] = {yq, m2};
        const T coef2[2] = {1, 1};
        adiag_all(x, y, m2, 2, in2, out2, coef2, nullptr, true);
        return;
      }
    }
    // delta = D_div u, e = nu delta + q; B^T u = M_q delta; g = M_q e
    divergence_plus<T>(x, x + nvc, x + 2 * nvc, a, b, delta, q, nu, m1, s, nb, bs);
    const T* in[2] = {delta, m1};
    T* out[2] = {yq, m2};
    const T coef[2] = {1, 1};
    if (Mc_w.val) {
      adiag_all(x, y, m2, 2, in, out, coef);
      return;
    }
    mq(2, in, out, coef);
    adiag_all(x, y, m2);
  }

  // y = A x; with h, the Horner step of h is applied to A x instead (y is scratch then)
  void apply_A(const T* x, T* y, const Horner<T>* h = nullptr) const {
    if constexpr (std::is_same<T, double>::value) {
      if (fused_div()) {
        div_band_x1<T>(x, x + nvc, x + 2 * nvc, a, b, nullptr, nu, Mc, f1, nullptr, s);
        const T* in1[1] = {f1};
        T* out1[1] = {m2};
        const T coef1[1] = {nu};
        adiag_all(x, y, m2, 1, in1, out1, coef1, h, true);
        return;
      }
    }
    divergence<T>(x, x + nvc, x + 2 * nvc, a, b, delta, s, nb, bs);
    const T* in[1] = {delta};
    T* out[1] = {m2};
    const T coef[1] = {nu};
    if (Mc_w.val) {
      adiag_all(x, y, m2, 1, in, out, coef, h);
      return;
    }
    mq(1, in, out, coef);
    adiag_all(x, y, m2, 0, nullptr, nullptr, nullptr, h);
  }

  // y = M_V x: L2 Gram matrix of the velocity basis, per component (mass (x) mass (x) mass with
  // the interior N-spline mass in the own direction)
  void mass_V(const T* x, T* y) const {
    PassArgs<T> j[3];
    for (int c = 0; c < 3; ++c)
      j[c] = job(x + c * nvc, M, 1, nullptr, nullptr, 0, comp(c), own_axis(c), tK + c * nvc);
    band_pass_multi<T>(j, 3, s);
    for (int c = 0; c < 3; ++c)
      j[c] = job(tK + c * nvc, Mc, 1, nullptr, nullptr, 0, comp(c), first_other(c), tS + c * nvc);
    band_pass_multi<T>(j, 3, s);
    for (int c = 0; c < 3; ++c)
      j[c] = job(tS + c * nvc, Mc, 1, nullptr, nullptr, 0, comp(c), second_other(c), y + c * nvc);
    band_pass_multi<T>(j, 3, s);
  }

  void apply_B(const T* q, T* yu) const {   // B q = D_div^T M_q q
    const T* in[1] = {q};
    T* out[1] = {m2};
    const T coef[1] = {1};
    mq(1, in, out, coef);
    div_transpose<T>(m2, a, b, yu, yu + nvc, yu + 2 * nvc, 0, s, nb, bs);
  }

  // B^T u = M_q D_div u; with h, the Horner step of h is applied to it instead
  void apply_Bt(const T* u, T* yq, const Horner<T>* h = nullptr) const {
    T* out[1] = {yq};
    const T coef[1] = {1};
    if constexpr (std::is_same<T, double>::value) {
      if (nb == 1 && b <= 512) {
        // the divergence and the pass along x1 in one launch (the same bits as two)
        div_band_x1<T>(u, u + nvc, u + 2 * nvc, a, b, nullptr, nu, Mc, f1, nullptr, s);
        const T* in1[1] = {f1};
        mq(1, in1, out, coef, h, true);
        return;
      }
    }
    divergence<T>(u, u + nvc, u + 2 * nvc, a, b, delta, s, nb, bs);
    const T* in[1] = {delta};
    mq(1, in, out, coef, h);
  }

  ModeArgs<T> mjob(const T* X, T* Y, const T* U, int n, int trans, Dims in, int axis,
                   const T* l1 = nullptr, const T* l2 = nullptr, const T* l3 = nullptr,
                   T scale = 1, T post = 1) const {
    ModeArgs<T> m{};
    m.X = X;
    m.Y = Y;
    m.U = U;
    m.ld = n;
    m.trans = trans;
    m.m = n;
    m.in = in;
    m.axis = axis;
    m.lam1 = l1;
    m.lam2 = l2;
    m.lam3 = l3;
    m.scale = scale;
    m.post = post;
    m.block = mode_block;
    return m;
  }

  // fast diagonalisation of the three diagonal blocks A_cc (App. A.4), all components per launch:
  // y_c = (U3 U2 U1) diag(1 / (2 nu (l1 + l2 + l3))) (U3 U2 U1)^T x_c, with (U, l) = (U_N, lam_N)
  // in the own direction of c and (U_T, lam_T) in the other two.
  // tensor t (0..2 velocity components, 3 pressure): canonical x -> canonical y
  // The pressure tensor (t = 3) takes three passes with the dense inverse of M-check instead:
  // (M-check^-1)^(x)3 is a Kronecker product of one dense matrix, so one rotation of the three
  // directions applies it (the eigenvector route U_T U_T^T needs six).
  void tc_fd(int t, const float* x, float* y) const {
    const Dims d = t < 3 ? comp(t) : Dims{b, b, b};
    pad_rows(x, d.n1, (int64_t)d.n2 * d.n3, tc_ld0[t], tc_p0[t], tc_bf16, s, nb, bs);
    const int passes = t < 3 ? 6 : 3;
    for (int st = 0; st < passes; ++st) {
      RmpPlan p = tc_plan[t * 6 + st];
      if (st == passes - 1) {
        p.args.Y = y;
        p.args.ybs = bs;
      }
      launch_rmp(p, tc_err, sms, s, tc_spin, tc_nsplit);
    }
  }

  // fused FP64 fast diagonalisation: selected, and every plane fits in shared memory
  bool fused_fd_ok() const {
    return fd_fused && eo_N >= 1 && eo_T >= 1 && fd_plane_smem(Dims{a, b, b}) > 0 &&
           fd_plane_smem(Dims{b, a, b}) > 0 && fd_plane_smem(Dims{b, b, b}) > 0;
  }

  void fd_V(const T* x, T* y) const {
    if (tc) {
      // the three components share each of the six tensor-core launches
      for (int c = 0; c < 3; ++c) {
        const Dims d = comp(c);
        pad_rows(reinterpret_cast<const float*>(x + c * nvc), d.n1, (int64_t)d.n2 * d.n3,
                 tc_ld0[c], tc_p0[c], tc_bf16, s, nb, bs);
      }
      for (int st = 0; st < 6; ++st) {
        RmpPlan p[3];
        const RmpPlan* pp[3];
        for (int c = 0; c < 3; ++c) {
          p[c] = tc_plan[c * 6 + st];
          if (st == 5) {
            p[c].args.Y = reinterpret_cast<float*>(y + c * nvc);
            p[c].args.ybs = bs;
          }
          pp[c] = &p[c];
        }
        launch_rmp_multi(pp, 3, tc_err, sms, s, tc_spin, tc_nsplit);
      }
      return;
    }
    const T* U[3][3];
    const T* L[3][3];
    int n[3][3];
    for (int c = 0; c < 3; ++c)
      for (int k = 0; k < 3; ++k) {
        const bool own = k == c;
        U[c][k] = own ? U_N : U_T;
        L[c][k] = own ? lam_N : lam_T;
        n[c][k] = own ? a : b;
      }
    if constexpr (std::is_same<T, double>::value) {
      if (fused_fd_ok()) {
        // three launches: (x1, x2) per plane, (x3, scaling, x3) per line group, (x2, x1) per
        // plane; the same bits as the six single-direction launches below
        FdPlaneArgs pa[3];
        FdLineArgs la[3];
        for (int c = 0; c < 3; ++c) {
          const int64_t o = c * nvc;
          const int e[3] = {c == 0 ? eo_N : eo_T, c == 1 ? eo_N : eo_T, c == 2 ? eo_N : eo_T};
          pa[c] = FdPlaneArgs{x + o, f1 + o, U[c][0], U[c][1], comp(c), e[0], e[1], 1.0};
          la[c] = FdLineArgs{f1 + o, f2 + o, U[c][2], comp(c), e[2], invd ? invd + o : nullptr,
                             L[c][0], L[c][1], L[c][2], 2 * nu, 1.0};
        }
        if (fd_plane_multi(pa, 3, 1, mode_block, fd_fused, s) && fd_line3_multi(la, 3, mode_block, s)) {
          for (int c = 0; c < 3; ++c) {
            pa[c].X = f2 + c * nvc;
            pa[c].Y = y + c * nvc;
          }
          if (fd_plane_multi(pa, 3, 0, mode_block, fd_fused, s)) return;
        }
        throw CudaError{cudaErrorInvalidValue, "fused fast diagonalisation rejected its jobs"};
      }
    }
    ModeArgs<T> j[3];
    const T* src;
    T* dst;
    // forward: U1^T, U2^T, U3^T (with the eigenvalue scaling); backward: U3, U2, U1
    const int axis_of[6] = {1, 2, 3, 3, 2, 1};
    const int trans_of[6] = {1, 1, 1, 0, 0, 0};
    for (int st = 0; st < 6; ++st) {
      for (int c = 0; c < 3; ++c) {
        const int64_t o = c * nvc;
        src = st == 0 ? x + o : ((st % 2) ? f1 + o : f2 + o);
        dst = st == 5 ? y + o : ((st % 2) ? f2 + o : f1 + o);
        const int k = axis_of[st] - 1;
        if (st == 2) {
          j[c] = mjob(src, dst, U[c][k], n[c][k], trans_of[st], comp(c), axis_of[st], L[c][0],
                      L[c][1], L[c][2], 2 * nu);
          j[c].invd = invd ? invd + o : nullptr;
        } else {
          j[c] = mjob(src, dst, U[c][k], n[c][k], trans_of[st], comp(c), axis_of[st]);
        }
        j[c].eo_he = (k == c) ? eo_N : eo_T;
      }
      mode_product_multi<T>(j, 3, s);
    }
  }

  void mode(const T* X, T* Y, const T* U, int n, int trans, Dims in, int axis, T post = 1,
            int eo = 0) const {
    ModeArgs<T> m = mjob(X, Y, U, n, trans, in, axis, nullptr, nullptr, nullptr, 1, post);
    m.eo_he = eo;
    mode_product<T>(m, s);
  }

  // pressure block: y = 2 nu (M-check^-1)^(x)3 x = 2 nu (U_T U_T^T)^(x)3 x
  void minv_Q(const T* x, T* y) const {
    // FP64: banded Cholesky line solves for large b (4(p + 1) FP64 flops per entry and direction
    // instead of 2b, exact up to rounding); for small b their sequential recurrence is
    // latency-bound and the dense route is faster. (In FP32 the tensor-core route below is
    // faster at every size: the line solves have one thread per line, a few warps per SM.)
    if constexpr (std::is_same<T, double>::value) {
      if (chol_lb && b >= 64) {
        ck(chol_solve_axis<T>(x, y, b, chol_p, 1, chol_lb, chol_inv, T(1), s, nb, bs), "chol");
        ck(chol_solve_axis<T>(y, y, b, chol_p, 2, chol_lb, chol_inv, T(1), s, nb, bs), "chol");
        ck(chol_solve_axis<T>(y, y, b, chol_p, 3, chol_lb, chol_inv, T(2) * nu, s, nb, bs),
           "chol");
        return;
      }
    }
    if (tc) {
      tc_fd(3, reinterpret_cast<const float*>(x), reinterpret_cast<float*>(y));
      return;
    }
    const Dims d{b, b, b};
    if constexpr (std::is_same<T, double>::value) {
      if (fused_fd_ok()) {
        FdPlaneArgs pa{x, f1, U_T, U_T, d, eo_T, eo_T, 1.0};
        FdLineArgs la{f1, f2, U_T, d, eo_T, nullptr, nullptr, nullptr, nullptr, 1.0, 1.0};
        if (fd_plane_multi(&pa, 1, 1, mode_block, fd_fused, s) && fd_line3_multi(&la, 1, mode_block, s)) {
          pa = FdPlaneArgs{f2, y, U_T, U_T, d, eo_T, eo_T, 2 * nu};
          if (fd_plane_multi(&pa, 1, 0, mode_block, fd_fused, s)) return;
        }
        throw CudaError{cudaErrorInvalidValue, "fused fast diagonalisation rejected its jobs"};
      }
    }
    mode(x, f1, U_T, b, 1, d, 1, 1, eo_T);
    mode(f1, f2, U_T, b, 1, d, 2, 1, eo_T);
    mode(f2, f1, U_T, b, 1, d, 3, 1, eo_T);
    mode(f1, f2, U_T, b, 0, d, 3, 1, eo_T);
    mode(f2, f1, U_T, b, 0, d, 2, 1, eo_T);
    mode(f1, y, U_T, b, 0, d, 1, 2 * nu, eo_T);
  }
};

// ---- quadrature-based forward operator (FP64) ---------------------------------------------------
// K [u; q] by matrix-free formation with global sum factorisation on the Gauss-Legendre grid of
// p + 2 points per element and direction (Sec. 5.3, the forward operator of Table 1's timings):
//   - the nine gradients d_d u_c and the pressure at the nq^3 points, by banded passes with the
//     value and derivative tables (N functions in a component's own direction, M elsewhere);
//   - pointwise, the weighted 2 nu eps(u) + q I and W div u (quad_stress);
//   - the transposed tables bring them back onto the test functions (a(u, v), b(v, q), b(u, .));
//   - the Nitsche face terms of sigma(u, v) (Sec. 3.2), which involve only the component itself
//     on each face (the other components' own-direction functions vanish there), as banded
//     Kronecker passes with Tface = T-check - K-check / 2 in the face-normal directions.
// Exact quadrature, so it equals the Kronecker operator to rounding (tests/test_gpu_quadrature).
struct QuadOps {
  int a = 0, b = 0, nq = 0;
  double nu = 0;
  int64_t nvc = 0, nvel = 0, n3 = 0;
  int band_block = 256;
  BandD<double> BN{}, DN{}, BM{}, DM{};       // nq x a, nq x a, nq x b, nq x b
  BandD<double> BNt{}, DNt{}, BMt{}, DMt{};   // transposes
  BandD<double> Tf{}, Mn{}, Mc{};             // b x b face part of T-check, a x a N mass, b x b
  const double* w = nullptr;                  // nq Gauss weights
  double* G = nullptr;                        // 9 x nq^3
  double* P = nullptr;                        // nq^3
  double *s1[2] = {nullptr, nullptr};         // x1 stage: nq * b * b
  double *s2[3] = {nullptr, nullptr, nullptr};  // x2 stage: nq * nq * b
  double *f1 = nullptr, *f2 = nullptr, *f3 = nullptr;   // face stage: component size
  cudaStream_t s = nullptr;

  Dims comp(int c) const {
    if (c == 0) return Dims{a, b, b};
    if (c == 1) return Dims{b, a, b};
    return Dims{b, b, a};
  }

  PassArgs<double> pj(const double* X0, const BandD<double>& D0, double c0, const double* X1,
                      const BandD<double>* D1, double c1, Dims in, int axis, double* Y,
                      const double* Z = nullptr, double cz = 0) const {
    PassArgs<double> p{};
    p.X0 = X0;
    p.D0 = D0;
    p.c0 = c0;
    p.X1 = X1;
    p.D1 = D1 ? *D1 : D0;
    p.c1 = c1;
    p.nterms = X1 ? 2 : 1;
    p.Z = Z;
    p.cz = cz;
    p.Y = Y;
    p.in = in;
    p.axis = axis;
    p.nb = 1;
    p.block = band_block;
    return p;
  }

  // table of component c (3 = pressure) in direction k (1..3): value or derivative
  const BandD<double>& tab(int c, int k, bool deriv, bool transposed) const {
    const bool own = c == k - 1;
    if (own) return deriv ? (transposed ? DNt : DN) : (transposed ? BNt : BN);
    return deriv ? (transposed ? DMt : DM) : (transposed ? BMt : BM);
  }

  void apply_K(const double* x, double* y) const {
    const double* q = x + nvel;
    PassArgs<double> j[3];
    // gradients d_d u_c at the points: x1 {value, derivative}, x2 {vv, vd, dv}, x3 {d1, d2, d3}
    for (int c = 0; c < 3; ++c) {
      const Dims e = comp(c);
      const double* u = x + c * nvc;
      const Dims d1{nq, e.n2, e.n3}, d2{nq, nq, e.n3};
      j[0] = pj(u, tab(c, 1, false, false), 1, nullptr, nullptr, 0, e, 1, s1[0]);
      j[1] = pj(u, tab(c, 1, true, false), 1, nullptr, nullptr, 0, e, 1, s1[1]);
      band_pass_multi<double>(j, 2, s);
      j[0] = pj(s1[0], tab(c, 2, false, false), 1, nullptr, nullptr, 0, d1, 2, s2[0]);   // v v
      j[1] = pj(s1[0], tab(c, 2, true, false), 1, nullptr, nullptr, 0, d1, 2, s2[1]);    // v d
      j[2] = pj(s1[1], tab(c, 2, false, false), 1, nullptr, nullptr, 0, d1, 2, s2[2]);   // d v
      band_pass_multi<double>(j, 3, s);
      double* g = G + (int64_t)3 * c * n3;
      j[0] = pj(s2[2], tab(c, 3, false, false), 1, nullptr, nullptr, 0, d2, 3, g);            // d/dx1
      j[1] = pj(s2[1], tab(c, 3, false, false), 1, nullptr, nullptr, 0, d2, 3, g + n3);       // d/dx2
      j[2] = pj(s2[0], tab(c, 3, true, false), 1, nullptr, nullptr, 0, d2, 3, g + 2 * n3);    // d/dx3
      band_pass_multi<double>(j, 3, s);
    }
    {  // pressure values at the points
      const Dims e{b, b, b}, d1{nq, b, b}, d2{nq, nq, b};
      j[0] = pj(q, BM, 1, nullptr, nullptr, 0, e, 1, s1[0]);
      band_pass_multi<double>(j, 1, s);
      j[0] = pj(s1[0], BM, 1, nullptr, nullptr, 0, d1, 2, s2[0]);
      band_pass_multi<double>(j, 1, s);
      j[0] = pj(s2[0], BM, 1, nullptr, nullptr, 0, d2, 3, P);
      band_pass_multi<double>(j, 1, s);
    }
    quad_stress(G, P, w, nq, nu, s);
    // Nitsche face terms into y_c: own direction N mass, then {Tface, M-check} in the first
    // other direction, then y_c = 2 nu (M-check (Tface t) + Tface (M-check t)) in the second
    for (int c = 0; c < 3; ++c) {
      const Dims e = comp(c);
      const int own = c + 1, o1 = c == 0 ? 2 : 1, o2 = c == 2 ? 2 : 3;
      j[0] = pj(x + c * nvc, Mn, 1, nullptr, nullptr, 0, e, own, f1);
      band_pass_multi<double>(j, 1, s);
      j[0] = pj(f1, Tf, 1, nullptr, nullptr, 0, e, o1, f2);
      j[1] = pj(f1, Mc, 1, nullptr, nullptr, 0, e, o1, f3);
      band_pass_multi<double>(j, 2, s);
      j[0] = pj(f2, Mc, 2 * nu, f3, &Tf, 2 * nu, e, o2, y + c * nvc);
      band_pass_multi<double>(j, 1, s);
    }
    // back onto the test functions: y_c += D1^T B2^T B3^T T_c1 + B1^T D2^T B3^T T_c2
    //                                       + B1^T B2^T D3^T T_c3
    for (int c = 0; c < 3; ++c) {
      const Dims e = comp(c);
      const Dims q3{nq, nq, nq}, d2{nq, nq, e.n3}, d1{nq, e.n2, e.n3};
      const double* t = G + (int64_t)3 * c * n3;
      j[0] = pj(t, tab(c, 3, false, true), 1, nullptr, nullptr, 0, q3, 3, s2[0]);
      j[1] = pj(t + n3, tab(c, 3, false, true), 1, nullptr, nullptr, 0, q3, 3, s2[1]);
      j[2] = pj(t + 2 * n3, tab(c, 3, true, true), 1, nullptr, nullptr, 0, q3, 3, s2[2]);
      band_pass_multi<double>(j, 3, s);
      const BandD<double>& B2t = tab(c, 2, false, true);
      j[0] = pj(s2[0], B2t, 1, nullptr, nullptr, 0, d2, 2, s1[0]);
      j[1] = pj(s2[1], tab(c, 2, true, true), 1, s2[2], &B2t, 1, d2, 2, s1[1]);
      band_pass_multi<double>(j, 2, s);
      const BandD<double>& B1t = tab(c, 1, false, true);
      double* yc = y + c * nvc;
      j[0] = pj(s1[0], tab(c, 1, true, true), 1, s1[1], &B1t, 1, d1, 1, yc, yc, 1);
      band_pass_multi<double>(j, 1, s);
    }
    {  // pressure rows: (B^T)^(x)3 W div u
      const Dims q3{nq, nq, nq}, d2{nq, nq, b}, d1{nq, b, b};
      j[0] = pj(P, BMt, 1, nullptr, nullptr, 0, q3, 3, s2[0]);
      band_pass_multi<double>(j, 1, s);
      j[0] = pj(s2[0], BMt, 1, nullptr, nullptr, 0, d2, 2, s1[0]);
      band_pass_multi<double>(j, 1, s);
      j[0] = pj(s1[0], BMt, 1, nullptr, nullptr, 0, d1, 1, y + nvel);
      band_pass_multi<double>(j, 1, s);
    }
  }
};

// ---- hyper-power recursion in precision T ------------------------------------------------------
template <typename T>
struct HyperPower {
  const Ops<T>* op = nullptr;
  // Optional second operator set (own workspace, own stream) for the pressure block. P_k is block
  // diagonal (Eq. 4.4, 4.5), so the velocity and pressure recursions are independent: apply()
  // runs them as two concurrent branches joined by events. Both branches launch the same kernels
  // on disjoint buffers, so the result is bit-identical to running them one after the other.
  const Ops<T>* opq = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool serial = false;   // run the branches one after the other (per-launch profiling)
  int order = 2;
  int schur = STOKES_SCHUR_INNER;
  struct VLevels {
    std::vector<T*> r, acc, t, u;   // velocity buffers per level 1..max_steps
  };
  VLevels vmain, vq;                  // velocity recursion; velocity solves inside the Schur block
  std::vector<T*> qr, qacc, qt, qu;   // pressure buffers per level
  T *bv = nullptr, *hv = nullptr;     // velocity buffers of the Schur approximation
  int64_t counts[4] = {0, 0, 0, 0};   // fd_V, minv_Q, A, (B + B^T)

  void V(const Ops<T>& o, const VLevels& L, int s, const T* x, T* y) {
    if (s == 0) {
      o.fd_V(x, y);
      ++counts[0];
      return;
    }
    T *r = L.r[s], *acc = L.acc[s], *t = L.t[s], *u = L.u[s];
    // Horner steps from r = acc = x; the first reads x directly
    for (int j = 1; j < order; ++j) {
      V(o, L, s - 1, j == 1 ? x : r, t);
      const Horner<T> h{j == 1 ? 1 : 2, r, acc, x};
      o.apply_A(t, u, &h);   // the step r, acc <- (r - A~ t, acc + r) in the last pass
      ++counts[2];
    }
    V(o, L, s - 1, acc, y);
  }

  int level_of(int m) const {
    if (schur == STOKES_SCHUR_NONE) return 0;
    return m == 1 ? 0 : m;
  }

  void Q(const Ops<T>& o, const VLevels& L, int m, const T* x, T* y) {
    if (m == 0) {
      o.minv_Q(x, y);
      ++counts[1];
      return;
    }
    T *r = qr[m], *acc = qacc[m], *t = qt[m], *u = qu[m];
    const int l = level_of(m);
    // Horner steps from r = acc = x; the first reads x directly
    for (int j = 1; j < order; ++j) {
      Q(o, L, m - 1, j == 1 ? x : r, t);
      o.apply_B(t, bv);          // A~_Q t = B^T P_{V,l}^-1 B t
      V(o, L, l, bv, hv);
      const Horner<T> h{j == 1 ? 1 : 2, r, acc, x};
      o.apply_Bt(hv, u, &h);   // the step r, acc <- (r - A~_Q t, acc + r) in the last pass
      ++counts[3];
    }
    Q(o, L, m - 1, acc, y);
  }

  void apply(int steps, const T* x, T* y) {
    if (!opq || serial) {
      V(*op, vmain, steps, x, y);
      Q(*op, vmain, steps, x + op->nvel, y + op->nvel);
      return;
    }
    ck(cudaEventRecord(ev_fork, op->s), "fork");
    ck(cudaStreamWaitEvent(opq->s, ev_fork, 0), "fork");
    V(*op, vmain, steps, x, y);
    Q(*opq, vq, steps, x + op->nvel, y + op->nvel);
    ck(cudaEventRecord(ev_join, opq->s), "join");
    ck(cudaStreamWaitEvent(op->s, ev_join, 0), "join");
  }
};

}  // namespace
}  // namespace shp

using namespace shp;

// The Arnoldi products w = K z of flexible GMRES in pair-of-FP32 arithmetic (k_pair.cu): the band
// matrices in centred form as pairs, pre-multiplied by the operator's nu and 2 nu, and the pair
// temporaries (item-major like every batched buffer, pitch ntot).
struct PairOps {
  bool on = false;
  int Ha = 0, Hb = 0;   // half widths: own-direction launch (K, M, M-check padded); the others
  PairBand K{}, M{}, Mc_a{}, Mc{}, nuMc{}, nu2Tc{};
  float2 nu{};
  float2 *tK = nullptr, *tM = nullptr, *tS = nullptr, *tR = nullptr;   // velocity size
  float2 *p1 = nullptr, *p2 = nullptr;   // two pressure tensors per item (delta and e passes)
  float2* m2 = nullptr;                  // M_q e
};

struct stokes_ctx {
  int n = 0, p = 0, a = 0, b = 0;
  double nu = 0, c_pen = 0;
  int64_t nvc = 0, nvel = 0, npres = 0, ntot = 0;
  stokes_opts opts{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Arena arena;
  Univariate uv;
  Ops<double> od;
  Ops<double> odq;                       // FP64 operators of the concurrent pressure branch
  cudaStream_t stream_q = nullptr;       // its stream (owned)
  Ops<float> of;
  Ops<float> ofq;                        // reduced-precision operators of the pressure branch
  QuadOps* quad = nullptr;               // quadrature-based forward operator (opts.forward)
  PairOps pk;                            // Arnoldi products in pair arithmetic (opts.outer)
  HyperPower<double> hd;
  HyperPower<float> hf;
  float *xf = nullptr, *yf = nullptr;    // reduced-precision preconditioner in/out
  double *zconst = nullptr, *ones = nullptr, *partials = nullptr, *dsc = nullptr;
  double* load1d = nullptr;              // three 1D factors of a separable load, 3 (b + 1)
  MinresState* st = nullptr;
  MinresState* st_host = nullptr;
  double* pinned = nullptr;              // small pinned host scratch
  double* pinned_multi = nullptr;        // 2 scalars per item (nrhs > 1)
  double* pinned_h = nullptr;            // Gram-Schmidt coefficients, restart + 2 per item
  // Krylov vectors
  double *kv[8] = {nullptr};
  double *V = nullptr, *Z = nullptr;     // FGMRES bases ((restart + 1) x ntot, restart x ntot)
  double *io_rhs = nullptr, *io_x = nullptr;
  int order = 2, steps = 0;
  int nb = 1;                     // right-hand sides (items) per vector, item stride ntot
  std::vector<double> ratios;
  std::string err;
  Profiler* prof = nullptr;
  bool prof_on = false;
  bool use_graphs = true;
  double* xi = nullptr;           // MINRES iterate (context-owned, so captured graphs are reusable)
  double* ratio_dev = nullptr;    // per-iteration convergence ratios
  std::map<int, cudaGraphExec_t> minres_graphs;
  std::map<int, int64_t> minres_graph_kernels;   // kernels per replay of each graph
  // FGMRES: one Arnoldi step's P and K applies captured per (order, steps) on fixed buffers
  std::map<int, cudaGraphExec_t> pk_graphs;
  std::map<int, int64_t> pk_graph_kernels;
  double *pk_in = nullptr, *pk_z = nullptr;   // nb * ntot each
  // set for the duration of stokes_solve_batch: replay existing graphs, capture no new one
  // (stream capture from the batch's concurrent host threads crashed the host process)
  bool no_capture = false;
  std::vector<RmpPlan> tc_plans, tc_plans_q;
  ~stokes_ctx() {
    delete quad;
    for (auto& kv : minres_graphs) cudaGraphExecDestroy(kv.second);
    for (auto& kv : pk_graphs) cudaGraphExecDestroy(kv.second);
    if (hd.ev_fork) cudaEventDestroy(hd.ev_fork);
    if (hd.ev_join) cudaEventDestroy(hd.ev_join);
    if (hf.ev_fork) cudaEventDestroy(hf.ev_fork);
    if (hf.ev_join) cudaEventDestroy(hf.ev_join);
  }
};

namespace {

// y = K x with the context's forward operator: banded Kronecker products (default) or the
// quadrature-based formation (opts.forward)
void apply_Kop(stokes_ctx* c, const double* x, double* y) {
  if (c->quad) c->quad->apply_K(x, y);
  else c->od.apply_K(x, y);
}

// ---- Arnoldi products in pair-of-FP32 arithmetic ----------------------------------------------
// largest |j - i| over the nonzero entries D(i, j) of a band matrix
int band_half(const Band& b) {
  int h = 0;
  for (int i = 0; i < b.rows; ++i)
    for (int w = 0; w < b.width; ++w)
      if (b.val[(size_t)i * b.width + w] != 0.0) h = std::max(h, std::abs(b.start[i] + w - i));
  return h;
}

// scale * D in the centred pair form of PairBand (half width H >= band_half(D), D square): each
// FP64 entry x split into hi = x rounded to FP32 and lo = (x - hi) rounded to FP32
PairBand upload_pair_band(Arena& ar, const Band& b, double scale, int H, cudaStream_t s) {
  PairBand d{};
  d.rows = b.rows;
  d.pitch = 2 * H + 2;
  const int rows8 = (b.rows + 7) / 8 * 8;
  std::vector<float2> cv((size_t)rows8 * d.pitch, make_float2(0.f, 0.f));
  for (int i = 0; i < b.rows; ++i)
    for (int w = 0; w < b.width; ++w) {
      const double v = b.val[(size_t)i * b.width + w];
      if (v == 0.0) continue;
      const int k = b.start[i] + w - i + H;
      if (k < 0 || k > 2 * H) throw SetupError{"band wider than its pair form"};
      const double x = scale * v;
      const float hi = (float)x;
      cv[(size_t)i * d.pitch + k] = make_float2(hi, (float)(x - (double)hi));
    }
  float2* dev = ar.alloc<float2>(cv.size());
  ck(cudaMemcpyAsync(dev, cv.data(), cv.size() * sizeof(float2), cudaMemcpyHostToDevice, s),
     "upload pair band");
  ck(cudaStreamSynchronize(s), "upload pair band");
  d.c = dev;
  return d;
}

size_t bsize(const stokes_ctx* c, int64_t per_item);

void init_pair(stokes_ctx* c, const Band& M, const Band& K, const Band& Mc, const Band& Tc) {
  PairOps& P = c->pk;
  P.on = false;
  if (c->opts.precision == STOKES_PREC_FP64 || c->opts.outer != STOKES_OUTER_PAIR ||
      c->opts.forward != STOKES_FORWARD_KRONECKER || c->b > 256)
    return;
  for (const Band* m : {&M, &K, &Mc, &Tc})
    if (m->rows != m->cols) return;
  P.Ha = std::max({band_half(K), band_half(M), band_half(Mc), 1});
  P.Hb = std::max({band_half(Mc), band_half(Tc), 1});
  if (P.Ha > 6 || P.Hb > 6) return;
  Arena& ar = c->arena;
  cudaStream_t s = c->stream;
  const double nu = c->nu;
  P.K = upload_pair_band(ar, K, 1.0, P.Ha, s);
  P.M = upload_pair_band(ar, M, 1.0, P.Ha, s);
  P.Mc_a = upload_pair_band(ar, Mc, 1.0, P.Ha, s);
  P.Mc = upload_pair_band(ar, Mc, 1.0, P.Hb, s);
  P.nuMc = upload_pair_band(ar, Mc, nu, P.Hb, s);
  P.nu2Tc = upload_pair_band(ar, Tc, 2.0 * nu, P.Hb, s);
  const float nh = (float)nu;
  P.nu = make_float2(nh, (float)(nu - (double)nh));
  P.tK = ar.alloc<float2>(bsize(c, c->nvel));
  P.tM = ar.alloc<float2>(bsize(c, c->nvel));
  P.tS = ar.alloc<float2>(bsize(c, c->nvel));
  P.tR = ar.alloc<float2>(bsize(c, c->nvel));
  P.p1 = ar.alloc<float2>(bsize(c, 2 * c->npres));
  P.p2 = ar.alloc<float2>(bsize(c, 2 * c->npres));
  P.m2 = ar.alloc<float2>(bsize(c, c->npres));
  P.on = true;
}

// y = K z for an FP32 z (every item) in pairs, the pass sequence of Ops::apply_K (grad-div
// factorisation through the pressure mass, sum factorisation of the diagonal blocks)
void pair_apply_K(stokes_ctx* c, const float* z, double* y) {
  const PairOps& P = c->pk;
  const Ops<double>& o = c->od;
  cudaStream_t s = c->stream;
  const int64_t nvc = c->nvc, nvel = c->nvel, npres = c->npres, bs = c->ntot;
  const int nb = c->nb;
  const Dims dq{c->b, c->b, c->b};
  ck(pair_div_x1(z, z + nvc, z + 2 * nvc, z + nvel, c->a, c->b, P.nu, P.Mc, P.Hb, P.p1,
                 P.p1 + npres, nb, bs, s), "pair divergence");
  auto job = [&](const void* X0, const PairBand& D0, const void* X1, const PairBand* D1,
                 int in_f32, Dims in, int axis, void* Y, int out_f64) {
    PairPass j{};
    j.X[0] = X0;
    j.D[0] = D0;
    j.X[1] = X1;
    j.D[1] = D1 ? *D1 : D0;
    j.nterms = X1 ? 2 : 1;
    j.in_f32 = in_f32;
    j.out_f64 = out_f64;
    j.Y = Y;
    j.in = in;
    j.axis = axis;
    j.nb = nb;
    j.bs = bs;
    return j;
  };
  PairPass j[kMaxPairJobs];
  // own direction: t_K = K u, t_M = M u; pressure mass of delta and e along x2
  for (int k = 0; k < 3; ++k) {
    const int64_t off = k * nvc;
    j[2 * k] = job(z + off, P.K, nullptr, nullptr, 1, o.comp(k), Ops<double>::own_axis(k),
                   P.tK + off, 0);
    j[2 * k + 1] = job(z + off, P.M, nullptr, nullptr, 1, o.comp(k), Ops<double>::own_axis(k),
                       P.tM + off, 0);
  }
  for (int k = 0; k < 2; ++k)
    j[6 + k] = job(P.p1 + k * npres, P.Mc_a, nullptr, nullptr, 0, dq, 2, P.p2 + k * npres, 0);
  ck(pair_pass_multi(j, 8, P.Ha, s), "pair pass");
  // first other direction: t_S = nu Mc t_K + 2 nu Tc t_M, t_R = Mc t_M; the pressure mass along
  // x3: B^T u = M_q delta into y, M_q e for the grad-div term
  for (int k = 0; k < 3; ++k) {
    const int64_t off = k * nvc;
    const int ax = Ops<double>::first_other(k);
    j[2 * k] = job(P.tK + off, P.nuMc, P.tM + off, &P.nu2Tc, 0, o.comp(k), ax, P.tS + off, 0);
    j[2 * k + 1] = job(P.tM + off, P.Mc, nullptr, nullptr, 0, o.comp(k), ax, P.tR + off, 0);
  }
  j[6] = job(P.p2, P.Mc, nullptr, nullptr, 0, dq, 3, y + nvel, 1);
  j[7] = job(P.p2 + npres, P.Mc, nullptr, nullptr, 0, dq, 3, P.m2, 0);
  ck(pair_pass_multi(j, 8, P.Hb, s), "pair pass");
  // second other direction: y_c = Mc t_S + 2 nu Tc t_R + D^T (M_q e) along the own direction
  for (int k = 0; k < 3; ++k) {
    const int64_t off = k * nvc;
    j[k] = job(P.tS + off, P.Mc, P.tR + off, &P.nu2Tc, 0, o.comp(k),
               Ops<double>::second_other(k), y + off, 1);
    j[k].g = P.m2;
    j[k].gaxis = Ops<double>::own_axis(k);
    j[k].gdims = dq;
  }
  ck(pair_pass_multi(j, 3, P.Hb, s), "pair pass");
}

// the Arnoldi product w = K z, z the FP64 copy of the preconditioner's output zf
void arnoldi_K(stokes_ctx* c, const float* zf, const double* z, double* w) {
  if (c->pk.on) pair_apply_K(c, zf, w);
  else apply_Kop(c, z, w);
}

thread_local std::string g_setup_error;

int fail(stokes_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg; else g_setup_error = msg;
  return code;
}

int cuda_fail(stokes_ctx* c, const CudaError& e) {
  return fail(c, STOKES_ERR_CUDA, std::string(e.what) + ": " + cudaGetErrorString(e.e));
}

void check_launch(const char* what) {
  ck(cudaGetLastError(), what);
}

template <typename T>
void alloc_workspace(stokes_ctx* c, Ops<T>& o);

template <typename T>
void init_ops(stokes_ctx* c, Ops<T>& o, const Band& M, const Band& K, const Band& Mc,
              const Band& Tc, const std::vector<double>& UN, const std::vector<double>& lN,
              const std::vector<double>& UT, const std::vector<double>& lT) {
  Arena& ar = c->arena;
  cudaStream_t s = c->stream;
  o.a = c->a;
  o.b = c->b;
  o.nu = (T)c->nu;
  o.nvc = c->nvc;
  o.nvel = c->nvel;
  o.npres = c->npres;
  o.s = s;
  o.M = upload_band<T>(ar, M, s);
  o.K = upload_band<T>(ar, K, s);
  o.Mc = upload_band<T>(ar, Mc, s);
  o.Tc = upload_band<T>(ar, Tc, s);
  if (std::is_same<T, double>::value) {
    o.Mc_nu = upload_band<T>(ar, scaled(Mc, c->nu), s);
    o.Tc_2nu = upload_band<T>(ar, scaled(Tc, 2.0 * c->nu), s);
  }
  {
    const Band Mcw = widen(Mc, K.width);
    if (Mcw.rows > 0 && o.K.cval && o.M.cval && o.K.half == o.M.half && 2 * o.K.half + 1 == K.width)
      o.Mc_w = upload_band<T>(ar, Mcw, s, o.K.half);
  }
  o.U_N = upload<T>(ar, UN, s);
  o.lam_N = upload<T>(ar, lN, s);
  o.U_T = upload<T>(ar, UT, s);
  o.lam_T = upload<T>(ar, lT, s);
  alloc_workspace(c, o);
}

// temporaries of one operator set (a second set lets a second stream run the same operators)
// entries of a buffer holding one item of `per_item` entries per right-hand side, item k at
// k * ntot (per_item <= ntot)
size_t bsize(const stokes_ctx* c, int64_t per_item) {
  return c->nb > 1 ? (size_t)(c->nb - 1) * (size_t)c->ntot + (size_t)per_item : (size_t)per_item;
}

template <typename T>
void alloc_workspace(stokes_ctx* c, Ops<T>& o) {
  Arena& ar = c->arena;
  const int64_t pres = c->npres, vel = c->nvel;
  const int64_t ping = std::max(vel, 2 * pres);   // all velocity components, or two pressures
  o.nb = c->nb;
  o.bs = c->ntot;
  o.tK = ar.alloc<T>(bsize(c, vel));
  o.tM = ar.alloc<T>(bsize(c, vel));
  o.tS = ar.alloc<T>(bsize(c, vel));
  o.tR = ar.alloc<T>(bsize(c, vel));
  o.f1 = ar.alloc<T>(bsize(c, ping));
  o.f2 = ar.alloc<T>(bsize(c, ping));
  o.delta = ar.alloc<T>(bsize(c, pres));
  o.m1 = ar.alloc<T>(bsize(c, pres));
  o.m2 = ar.alloc<T>(bsize(c, pres));
}

int rup(int x, int m) { return (x + m - 1) / m * m; }

// Tensor-core fast diagonalisation: padded operators (rows npad = n rounded to 16, row pitch
// kpad = n rounded to one 128-byte chunk), shared by both operator sets; per set (main, and the
// pressure branch's when it has one) its own rotation buffers and 4 x 6 TMA plans.
void init_tc_plans(stokes_ctx* c, Ops<float>& o, std::vector<RmpPlan>& plans, void* const* op,
                   const int* npad_of, const int* kpad_of, int kind);

void init_tc(stokes_ctx* c, const Dense& UN, const std::vector<double>& lN, const Dense& UT,
             const std::vector<double>& lT, int kind) {
  const int a = c->a, b = c->b;
  if (!rmp_supported(kind, a, a) || !rmp_supported(kind, b, b)) return;   // CUDA-core fallback
  const bool bf = kind == kMmaBF16;
  const int elem = bf ? 2 : 4;
  const int kchunk = 128 / elem;
  const int align = 16 / elem;
  Arena& ar = c->arena;
  cudaStream_t s = c->stream;
  // padded operators: op[0] = U_N^T, op[1] = U_N, op[2] = U_T^T, op[3] = U_T (Op[i][j] rows),
  // op[4] = M-check^-1 = U_T U_T^T (U_T^T M-check U_T = I), formed in FP64
  Dense Minv(b, b);
  for (int i = 0; i < b; ++i)
    for (int j = 0; j < b; ++j) {
      double acc = 0.0;
      for (int k = 0; k < b; ++k) acc += UT(i, k) * UT(j, k);
      Minv(i, j) = acc;
    }
  const Dense* srcs[5] = {&UN, &UN, &UT, &UT, &Minv};
  const bool transp[5] = {true, false, true, false, false};
  void* op[5];
  int npad_of[5], kpad_of[5];
  for (int k = 0; k < 5; ++k) {
    const int n = srcs[k]->rows;
    const int npad = rup(n, 16), kpad = rup(n, kchunk);
    npad_of[k] = npad;
    kpad_of[k] = kpad;
    std::vector<float> hf((size_t)npad * kpad, 0.f);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        hf[(size_t)i * kpad + j] = (float)(transp[k] ? (*srcs[k])(j, i) : (*srcs[k])(i, j));
    if (!bf) {
      // TF32 operands: round each entry to the nearest TF32 value (ties away from zero), as
      // the device rounds the data operands; the tensor cores would otherwise truncate
      for (float& v : hf) {
        uint32_t u;
        std::memcpy(&u, &v, 4);
        u = (u + 0x1000u) & 0xFFFFE000u;
        std::memcpy(&v, &u, 4);
      }
    }
    if (bf) {
      std::vector<uint16_t> hb(hf.size());
      for (size_t i = 0; i < hf.size(); ++i) {   // round to nearest even
        uint32_t u;
        std::memcpy(&u, &hf[i], 4);
        u += 0x7FFF + ((u >> 16) & 1);
        hb[i] = (uint16_t)(u >> 16);
      }
      op[k] = ar.alloc<uint16_t>(hb.size());
      ck(cudaMemcpyAsync(op[k], hb.data(), hb.size() * 2, cudaMemcpyHostToDevice, s), "op");
    } else {
      op[k] = ar.alloc<float>(hf.size());
      ck(cudaMemcpyAsync(op[k], hf.data(), hf.size() * 4, cudaMemcpyHostToDevice, s), "op");
    }
    ck(cudaStreamSynchronize(s), "op");
  }
  init_tc_plans(c, c->of, c->tc_plans, op, npad_of, kpad_of, kind);
  if (c->ofq.s) init_tc_plans(c, c->ofq, c->tc_plans_q, op, npad_of, kpad_of, kind);
}

void init_tc_plans(stokes_ctx* c, Ops<float>& o, std::vector<RmpPlan>& plans, void* const* op,
                   const int* npad_of, const int* kpad_of, int kind) {
  const int b = c->b;
  const bool bf = kind == kMmaBF16;
  const int elem = bf ? 2 : 4;
  const int align = 16 / elem;
  Arena& ar = c->arena;
  cudaStream_t s = c->stream;
  // elements per rotation slot: one tensor (the largest rotated layout) of every item
  const int nb = c->nb;
  const size_t slot = (size_t)rup(rup(b, align) * b * b, 64) * nb;
  uint8_t* P0 = reinterpret_cast<uint8_t*>(ar.alloc<float>(slot * 4 * elem / 4 + 64));
  uint8_t* F1 = reinterpret_cast<uint8_t*>(ar.alloc<float>(slot * 4 * elem / 4 + 64));
  uint8_t* F2 = reinterpret_cast<uint8_t*>(ar.alloc<float>(slot * 4 * elem / 4 + 64));
  ck(cudaMemsetAsync(P0, 0, slot * 4 * elem, s), "memset");
  ck(cudaMemsetAsync(F1, 0, slot * 4 * elem, s), "memset");
  ck(cudaMemsetAsync(F2, 0, slot * 4 * elem, s), "memset");
  o.tc_err = ar.alloc<int>(1);
  ck(cudaMemsetAsync(o.tc_err, 0, sizeof(int), s), "memset");
  int dev = 0;
  ck(cudaGetDevice(&dev), "device");
  ck(cudaDeviceGetAttribute(&o.sms, cudaDevAttrMultiProcessorCount, dev), "sms");
  plans.assign(24, RmpPlan{});
  for (int t = 0; t < 4; ++t) {
    const Dims d = t < 3 ? o.comp(t) : Dims{b, b, b};
    const int ext[3] = {d.n1, d.n2, d.n3};
    const bool own[3] = {t == 0, t == 1, t == 2};
    const float* lam[3];
    for (int k = 0; k < 3; ++k) lam[k] = own[k] ? o.lam_N : o.lam_T;
    uint8_t* bufs_in[6] = {P0, F1, F2, F1, F2, F1};
    uint8_t* bufs_out[6] = {F1, F2, F1, F2, F1, nullptr};
    if (t == 3) bufs_out[2] = nullptr;   // pressure: three passes, the third one canonical
    o.tc_p0[t] = P0 + (size_t)t * slot * elem;
    o.tc_ld0[t] = rup(ext[0], align);
    const int last = t < 3 ? 5 : 2;
    for (int st = 0; st <= last; ++st) {
      const int ax = st % 3;   // contracted direction: x1, x2, x3, x1, x2, x3
      const int e1 = ext[ax], e2 = ext[(ax + 1) % 3], e3 = ext[(ax + 2) % 3];
      const bool fwd = st < 3;
      // operator index: velocity own direction uses U_N, the other directions U_T; the
      // pressure uses the dense inverse of M-check in each of its three passes
      const int base_op = (t < 3 && own[ax]) ? 0 : 2;
      const int opk = t == 3 ? 4 : base_op + (fwd ? 0 : 1);
      RmpPlan& p = plans[t * 6 + st];
      p.kind = kind;
      p.out_bf16 = bf && st < last;
      RmpArgs& ra = p.args;
      ra.R = e2 * e3;
      ra.K = e1;
      ra.m = e1;
      ra.npad = npad_of[opk];
      ra.e2 = e2;
      ra.e3 = e3;
      ra.ldy = st < last ? rup(e2, align) : e2;
      ra.round_tf32 = (!bf && st < last) ? 1 : 0;
      ra.idesc = rmp_idesc(kind, ra.npad);
      ra.scale = (float)(2.0 * c->nu);
      ra.post = 1.f;
      if (st == 2 && t < 3) {
        ra.lam_j2 = lam[0];
        ra.lam_j3 = lam[1];
        ra.lam_i = lam[2];
      }
      if (st == last && t == 3) ra.post = (float)(2.0 * c->nu);
      ra.Y = bufs_out[st] ? (void*)(bufs_out[st] + (size_t)t * slot * elem) : nullptr;
      // items: the rotated output of item k follows item k - 1's (e3 * m rows of pitch ldy,
      // the next step's input rows); the final step's output is canonical (set at launch)
      ra.nb = nb;
      ra.ybs = (int64_t)ra.ldy * e3 * ra.m;
      const void* in = bufs_in[st] + (size_t)t * slot * elem;
      if (!make_map(p.map_x, in, kind, e1, (int64_t)e2 * e3 * nb, rup(e1, align), 128) ||
          !make_map(p.map_op, op[opk], kind, e1, ra.npad, kpad_of[opk], ra.npad))
        throw SetupError{"tensor map encoding failed"};
    }
  }
  ck(cudaStreamSynchronize(s), "memset");
  o.tc_plan = plans.data();
  o.tc_bf16 = bf;
  o.tc = true;
}

template <typename T>
void alloc_levels(stokes_ctx* c, typename HyperPower<T>::VLevels& L) {
  const int n = c->opts.max_steps;
  L.r.assign(n + 1, nullptr);
  L.acc.assign(n + 1, nullptr);
  L.t.assign(n + 1, nullptr);
  L.u.assign(n + 1, nullptr);
  for (int l = 1; l <= n; ++l) {
    L.r[l] = c->arena.alloc<T>(bsize(c, c->nvel));
    L.acc[l] = c->arena.alloc<T>(bsize(c, c->nvel));
    L.t[l] = c->arena.alloc<T>(bsize(c, c->nvel));
    L.u[l] = c->arena.alloc<T>(bsize(c, c->nvel));
  }
}

// opq: operator set of the concurrent pressure branch, or null (one stream)
template <typename T>
void init_hp(stokes_ctx* c, HyperPower<T>& h, const Ops<T>& o, const Ops<T>* opq) {
  Arena& ar = c->arena;
  h.op = &o;
  h.opq = opq;
  h.schur = c->opts.schur;
  const int L = c->opts.max_steps;
  alloc_levels<T>(c, h.vmain);
  if (opq) {
    alloc_levels<T>(c, h.vq);
    ck(cudaEventCreateWithFlags(&h.ev_fork, cudaEventDisableTiming), "event");
    ck(cudaEventCreateWithFlags(&h.ev_join, cudaEventDisableTiming), "event");
  }
  h.qr.assign(L + 1, nullptr);
  h.qacc.assign(L + 1, nullptr);
  h.qt.assign(L + 1, nullptr);
  h.qu.assign(L + 1, nullptr);
  for (int l = 1; l <= L; ++l) {
    h.qr[l] = ar.alloc<T>(bsize(c, c->npres));
    h.qacc[l] = ar.alloc<T>(bsize(c, c->npres));
    h.qt[l] = ar.alloc<T>(bsize(c, c->npres));
    h.qu[l] = ar.alloc<T>(bsize(c, c->npres));
  }
  if (L > 0) {
    h.bv = ar.alloc<T>(bsize(c, c->nvel));
    h.hv = ar.alloc<T>(bsize(c, c->nvel));
  }
}

bool reduced(const stokes_ctx* c) { return c->opts.precision != STOKES_PREC_FP64; }

// y = P_s^-1 x in the context's preconditioner precision (x, y: FP64 device vectors)
void apply_prec(stokes_ctx* c, int order, int steps, const double* x, double* y) {
  if (!reduced(c)) {
    c->hd.order = order;
    c->hd.apply(steps, x, y);
  } else {
    const int64_t n = (int64_t)c->nb * c->ntot;   // every item
    to_float(x, c->xf, n, c->stream);
    c->hf.order = order;
    c->hf.apply(steps, c->xf, c->yf);
    to_double(c->yf, y, n, c->stream);
  }
}

double read_scalar(stokes_ctx* c, const double* d) {
  ck(cudaMemcpyAsync(c->pinned, d, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "read");
  ck(cudaStreamSynchronize(c->stream), "sync");
  return c->pinned[0];
}

// zero-mean pressure (the constant pressure spans the null space of K, Sec. 3.2)
void normalize_pressure(stokes_ctx* c, double* x) {
  double* q = x + c->nvel;
  dot<double>(q, c->ones, c->npres, c->partials, c->dsc + 0, c->stream);
  axpy_dev(c->dsc + 0, -1.0, c->zconst, q, c->npres, c->stream);
}

// true relative residual ||f - K x|| / ||f||
double true_residual(stokes_ctx* c, const double* f, const double* x, double* tmp) {
  apply_Kop(c, x, tmp);
  axpby<double>(1.0, f, -1.0, tmp, c->ntot, c->stream);
  dot<double>(tmp, tmp, c->ntot, c->partials, c->dsc + 1, c->stream);
  dot<double>(f, f, c->ntot, c->partials, c->dsc + 2, c->stream);
  ck(cudaMemcpyAsync(c->pinned, c->dsc + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                     c->stream), "read");
  ck(cudaStreamSynchronize(c->stream), "sync");
  const double rr = c->pinned[0], ff = c->pinned[1];
  return ff > 0 ? std::sqrt(rr / ff) : std::sqrt(rr);
}

// One MINRES iteration (Paige-Saunders recurrences with all scalars on the device). The buffer
// roles rotate with period two, so two consecutive iterations form a fixed launch sequence.
void minres_iteration(stokes_ctx* c, double* vold, double* v, double* z, double* zn, double* wold,
                      double* w, double* Kz, double* x) {
  const int64_t n = c->ntot;
  cudaStream_t s = c->stream;
  minres_scale_z(z, c->st, n, s);
  apply_Kop(c, z, Kz);
  dot<double>(Kz, z, n, c->partials, &c->st->delta, s);
  minres_lanczos(Kz, v, vold, c->st, n, s);            // v_new over v_old
  apply_prec(c, c->order, c->steps, vold, zn);
  dot<double>(zn, vold, n, c->partials, &c->st->gg, s);
  minres_scalars(c->st, s);
  minres_update(z, wold, w, x, c->st, n, s);           // w_new over w_old, x += ...
}

void minres_pair(stokes_ctx* c) {
  double** k = c->kv;
  // roles: vold, v, z, zn, wold, w; Kz = kv[4]; iterate into the context buffer xi
  minres_iteration(c, k[0], k[1], k[2], k[3], k[5], k[6], k[4], c->xi);
  minres_iteration(c, k[1], k[0], k[3], k[2], k[6], k[5], k[4], c->xi);
}

bool profiling_active(stokes_ctx* c) { return c->prof_on; }

// Captures what `record` enqueues on stream s into an instantiated graph and returns it with
// the number of kernels it replays. One capture at a time in the process (stream capture from
// several host threads at once crashed the host process, see stokes_solve_batch); the kernels
// enqueued while capturing are not counted as launches (they run when the graph is replayed).
std::mutex g_capture_mutex;

template <typename F>
cudaGraphExec_t capture_graph(cudaStream_t s, F&& record, int64_t* kernels) {
  std::lock_guard<std::mutex> lock(g_capture_mutex);
  cudaGraph_t g = nullptr;
  set_capturing(true);
  try {
    ck(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "capture");
    record();
    ck(cudaStreamEndCapture(s, &g), "capture");
  } catch (...) {
    set_capturing(false);
    throw;
  }
  set_capturing(false);
  size_t nn = 0;
  ck(cudaGraphGetNodes(g, nullptr, &nn), "graph nodes");
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) ck(cudaGraphGetNodes(g, nodes.data(), &nn), "graph nodes");
  int64_t k = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    ck(cudaGraphNodeGetType(nd, &t), "graph node");
    if (t == cudaGraphNodeTypeKernel) ++k;
  }
  cudaGraphExec_t exec = nullptr;
  ck(cudaGraphInstantiate(&exec, g, 0), "instantiate");
  cudaGraphDestroy(g);
  *kernels = k;
  return exec;
}

int run_minres(stokes_ctx* c, const double* f, double tol, double* x, int* iters) {
  const int64_t n = c->ntot;
  cudaStream_t s = c->stream;
  double** k = c->kv;
  fill_zero(c->xi, n * sizeof(double), s);
  fill_zero(k[0], n * sizeof(double), s);
  fill_zero(k[5], n * sizeof(double), s);
  fill_zero(k[6], n * sizeof(double), s);
  copy_async(k[1], f, n * sizeof(double), s);
  MinresState* h = c->st_host;
  std::memset(h, 0, sizeof(MinresState));
  h->tol = tol;
  h->ratios = c->ratio_dev;
  h->cap = c->opts.maxit;
  ck(cudaMemcpyAsync(c->st, h, sizeof(MinresState), cudaMemcpyHostToDevice, s), "state");
  apply_prec(c, c->order, c->steps, k[1], k[2]);
  dot<double>(k[2], k[1], n, c->partials, &c->st->gg, s);
  minres_init(c->st, s);
  check_launch("minres init");
  ck(cudaMemcpyAsync(h, c->st, sizeof(MinresState), cudaMemcpyDeviceToHost, s), "state");
  ck(cudaStreamSynchronize(s), "sync");
  c->ratios.clear();
  int rc = STOKES_OK;
  if (h->status != 0) {
    rc = h->status;
  } else if (!h->done) {
    // two iterations per replay of a captured graph (or per direct launch sequence when a
    // profiler is recording events or graphs are disabled)
    cudaGraphExec_t exec = nullptr;
    const int gkey = c->order * 16 + c->steps;
    const bool use_graph = c->use_graphs && !profiling_active(c) &&
                           !(c->no_capture && c->minres_graphs.find(gkey) == c->minres_graphs.end());
    if (use_graph) {
      const int key = gkey;
      auto it = c->minres_graphs.find(key);
      if (it == c->minres_graphs.end()) {
        int64_t k = 0;
        exec = capture_graph(s, [&] { minres_pair(c); }, &k);
        c->minres_graphs[key] = exec;
        c->minres_graph_kernels[key] = k;
      } else {
        exec = it->second;
      }
    }
    const int64_t graph_kernels = use_graph ? c->minres_graph_kernels[c->order * 16 + c->steps] : 0;
    for (int pair = 0; 2 * pair < c->opts.maxit; ++pair) {
      if (use_graph) {
        ck(cudaGraphLaunch(exec, s), "graph launch");
        launch_add(graph_kernels);
      } else {
        minres_pair(c);
      }
      check_launch("minres iteration");
      ck(cudaMemcpyAsync(h, c->st, sizeof(MinresState), cudaMemcpyDeviceToHost, s), "state");
      ck(cudaStreamSynchronize(s), "sync");
      if (h->status != 0 || h->done) break;
    }
    if (h->status != 0) rc = h->status;
    else if (!h->done) rc = STOKES_ERR_MAXIT;
  }
  *iters = h->iter;
  if (h->iter > 0) {
    c->ratios.resize(std::min(h->iter, c->opts.maxit));
    ck(cudaMemcpyAsync(c->ratios.data(), c->ratio_dev, c->ratios.size() * sizeof(double),
                       cudaMemcpyDeviceToHost, s), "ratios");
  }
  copy_async(x, c->xi, n * sizeof(double), s);
  ck(cudaStreamSynchronize(s), "sync");
  return rc;
}

// One Arnoldi step's products, for every item: z = P_s^-1 v, then w = K z. With graphs enabled
// (and no profiler recording) the two applies are captured once per (order, steps) on fixed
// buffers (v copied in, z copied out, w always the context's first Krylov vector) and replayed,
// so the host issues three operations instead of every kernel of the recursion. Same kernels in
// the same order: the result does not depend on the path.
void pk_apply(stokes_ctx* c, const double* v, double* z, double* w) {
  cudaStream_t s = c->stream;
  const size_t bytes = (size_t)c->nb * c->ntot * sizeof(double);
  const int key = c->order * 16 + c->steps;
  auto it = c->pk_graphs.find(key);
  if (!c->use_graphs || profiling_active(c) || !c->pk_in || w != c->kv[0] ||
      (c->no_capture && it == c->pk_graphs.end())) {
    apply_prec(c, c->order, c->steps, v, z);
    arnoldi_K(c, c->yf, z, w);
    return;
  }
  cudaGraphExec_t exec = nullptr;
  if (it == c->pk_graphs.end()) {
    int64_t k = 0;
    exec = capture_graph(s, [&] {
      apply_prec(c, c->order, c->steps, c->pk_in, c->pk_z);
      arnoldi_K(c, c->yf, c->pk_z, w);
    }, &k);
    c->pk_graphs[key] = exec;
    c->pk_graph_kernels[key] = k;
  } else {
    exec = it->second;
  }
  copy_async(c->pk_in, v, bytes, s);
  ck(cudaGraphLaunch(exec, s), "graph launch");
  launch_add(c->pk_graph_kernels[key]);
  copy_async(z, c->pk_z, bytes, s);
}

// Gram-Schmidt step of flexible GMRES for every item k with active[k]: w_k (= K z_j of item k,
// item k at w + k ntot) is orthogonalised against its basis vectors V_0 .. V_j (item k of V_i at
// c->V + i N + k ntot) by classical Gram-Schmidt applied twice, in one sweep over the basis:
//   c = V^T w and d = V^T v_j (the new column of the Gram matrix G = V^T V, which is the identity
//   up to the rounding of the basis) and <w, w> come from one fused reduction;
//   the two passes' coefficients are h = c + (c - G c): the second pass's products
//   V^T (w - V c) equal c - G c exactly in real arithmetic, so the reduction that forms them is
//   replaced by the Gram matrix the earlier sweeps built (one column per step);
//   ||w - V h||^2 = <w, w> - 2 h.c + h^T G h, and V_{j+1} = (w - V h) / ||w - V h|| is written by
//   one fused update-and-divide sweep.
// This is the one-reduction form of reorthogonalised classical Gram-Schmidt (the Gram-matrix
// correction of the low-synchronisation Gram-Schmidt methods, Swirydowicz, Langou, Ananthan, Yang
// and Thomas, 2020): two sweeps over the basis per step instead of four, one host read.
// When the update cancels all but 1e-6 of <w, w> (a near breakdown, where the expanded norm
// loses its accuracy), the vector is updated first and its norm taken by a dot product.
// gram[k] ((m + 1)^2, row-major) holds item k's Gram matrix for the current cycle; cols[k][0..j]
// receives item k's Hessenberg column h, hn[k] h_{j+1,j}; bad[k] is set when a value is not
// finite. Scalars per item k at c->dsc + k ds: c, d, <w, w> from +8, h_{j+1,j} at +7, a dot at +6;
// h is staged through c->pinned_h to +8 + (m + 2).
void arnoldi_gs(stokes_ctx* c, int j, const std::vector<char>& active, double* w,
                std::vector<std::vector<double>>& gram, std::vector<std::vector<double>>& cols,
                std::vector<double>& hn, std::vector<char>& bad) {
  const int nb = c->nb;
  const int64_t n = c->ntot, N = (int64_t)nb * n;
  cudaStream_t s = c->stream;
  const int m = c->opts.restart;
  const int mg = m + 1;
  const size_t ds = 16 + 2 * (size_t)(m + 2);
  const int nv = j + 1;
  auto base = [&](int k) { return c->dsc + (size_t)k * ds; };
  std::vector<double> hs((size_t)nb * ds);
  auto read_all = [&]() {
    ck(cudaMemcpyAsync(hs.data(), c->dsc, hs.size() * sizeof(double), cudaMemcpyDeviceToHost, s),
       "read");
    ck(cudaStreamSynchronize(s), "sync");
  };
  for (int k = 0; k < nb; ++k)
    if (active[k])
      multi_dot2(c->V + k * n, N, nv, w + k * n, c->V + (int64_t)j * N + k * n, n,
                 c->partials + kDotScratch, base(k) + 8, s);
  check_launch("fgmres arnoldi");
  read_all();
  std::vector<char> explicit_norm(nb, 0);
  bool any_explicit = false;
  for (int k = 0; k < nb; ++k) {
    if (!active[k]) continue;
    const double* cv = hs.data() + (size_t)k * ds + 8;
    const double* dv = cv + nv;
    const double ww = dv[nv];
    std::vector<double>& G = gram[k];
    for (int i = 0; i <= j; ++i) G[(size_t)i * mg + j] = G[(size_t)j * mg + i] = dv[i];
    std::vector<double>& h = cols[k];
    h.assign(nv, 0.0);
    for (int i = 0; i < nv; ++i) {
      double gc = 0.0;
      for (int l = 0; l < nv; ++l) gc += G[(size_t)i * mg + l] * cv[l];
      h[i] = cv[i] + (cv[i] - gc);
    }
    double hc = 0.0, hgh = 0.0;
    for (int i = 0; i < nv; ++i) {
      hc += h[i] * cv[i];
      double gh = 0.0;
      for (int l = 0; l < nv; ++l) gh += G[(size_t)i * mg + l] * h[l];
      hgh += h[i] * gh;
    }
    const double s2 = ww - 2.0 * hc + hgh;
    bool finite = std::isfinite(ww) && std::isfinite(s2);
    for (int i = 0; i < nv && finite; ++i) finite = std::isfinite(h[i]);
    if (!finite) {
      bad[k] = 1;
      continue;
    }
    double* hp = c->pinned_h + (size_t)k * (m + 2);
    for (int i = 0; i < nv; ++i) hp[i] = h[i];
    double* hdev = base(k) + 8 + (m + 2);
    ck(cudaMemcpyAsync(hdev, hp, nv * sizeof(double), cudaMemcpyHostToDevice, s), "h");
    if (s2 > 1e-6 * ww) {
      const double hv = std::sqrt(s2);
      hn[k] = hv;
      hp[m + 1] = hv;
      ck(cudaMemcpyAsync(base(k) + 7, hp + m + 1, sizeof(double), cudaMemcpyHostToDevice, s),
         "h");
      multi_axpy_div(c->V + k * n, N, nv, hdev, -1.0, w + k * n, base(k) + 7,
                     c->V + (int64_t)nv * N + k * n, n, s);
    } else {   // w -= V h, then its norm from a dot product
      explicit_norm[k] = 1;
      any_explicit = true;
      multi_axpy(c->V + k * n, N, nv, hdev, -1.0, w + k * n, n, s);
      dot<double>(w + k * n, w + k * n, n, c->partials, base(k) + 6, s);
    }
  }
  if (!any_explicit) return;
  read_all();
  for (int k = 0; k < nb; ++k) {
    if (!explicit_norm[k]) continue;
    const double h = std::sqrt(hs[(size_t)k * ds + 6]);
    if (!std::isfinite(h)) {
      bad[k] = 1;
      continue;
    }
    hn[k] = h;
    if (h > 0.0) {
      double* hp = c->pinned_h + (size_t)k * (m + 2);
      hp[m + 1] = h;
      ck(cudaMemcpyAsync(base(k) + 7, hp + m + 1, sizeof(double), cudaMemcpyHostToDevice, s),
         "h");
      scale_inv_dev(base(k) + 7, w + k * n, c->V + (int64_t)nv * N + k * n, n, s);
    }
  }
}

// Right-preconditioned flexible GMRES (Saad 1993): classical Gram-Schmidt with a second pass
// only where the first cancels (arnoldi_gs), Givens rotations on the host.
int run_fgmres(stokes_ctx* c, const double* f, double tol, double* x, int* iters) {
  const int64_t n = c->ntot;
  cudaStream_t s = c->stream;
  const int m = c->opts.restart;
  double* w = c->kv[0];
  double* r = c->kv[1];
  double* hdev = c->dsc + 8;           // solution coefficients y at the end of a cycle
  fill_zero(x, n * sizeof(double), s);
  c->ratios.clear();
  dot<double>(f, f, n, c->partials, c->dsc + 3, s);
  const double fnorm = std::sqrt(read_scalar(c, c->dsc + 3));
  if (!std::isfinite(fnorm)) return STOKES_ERR_NONFINITE;
  if (fnorm == 0.0) {
    *iters = 0;
    return STOKES_OK;
  }
  int it = 0;
  copy_async(r, f, n * sizeof(double), s);
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  std::vector<std::vector<double>> cols(1), gram(1, std::vector<double>((size_t)(m + 1) * (m + 1)));
  std::vector<double> hnv(1);
  std::vector<char> act(1, 1), bad(1, 0);
  while (it < c->opts.maxit) {
    dot<double>(r, r, n, c->partials, c->dsc + 4, s);
    const double beta = std::sqrt(read_scalar(c, c->dsc + 4));
    if (!std::isfinite(beta)) return STOKES_ERR_NONFINITE;
    if (beta == 0.0) {
      *iters = it;
      return STOKES_OK;
    }
    c->pinned[0] = beta;
    ck(cudaMemcpyAsync(c->dsc + 5, c->pinned, sizeof(double), cudaMemcpyHostToDevice, s), "beta");
    scale_inv_dev(c->dsc + 5, r, c->V, n, s);
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k_used = 0;
    bool done = false;
    for (int j = 0; j < m; ++j) {
      double* Vj = c->V + (int64_t)j * n;
      double* Zj = c->Z + (int64_t)j * n;
      pk_apply(c, Vj, Zj, w);
      arnoldi_gs(c, j, act, w, gram, cols, hnv, bad);   // writes V_{j+1}
      if (bad[0]) return STOKES_ERR_NONFINITE;
      const double hn = hnv[0];
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = cols[0][i];
      H[(size_t)(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * H[(size_t)i * m + j] + sn[i] * H[(size_t)(i + 1) * m + j];
        H[(size_t)(i + 1) * m + j] = -sn[i] * H[(size_t)i * m + j] + cs[i] * H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = t;
      }
      const double hjj = H[(size_t)j * m + j], hj1 = H[(size_t)(j + 1) * m + j];
      const double den = std::hypot(hjj, hj1);
      if (den == 0.0) return STOKES_ERR_BREAKDOWN;
      cs[j] = hjj / den;
      sn[j] = hj1 / den;
      H[(size_t)j * m + j] = den;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++it;
      k_used = j + 1;
      const double ratio = std::fabs(g[j + 1]) / fnorm;
      c->ratios.push_back(ratio);
      if (ratio <= tol || it >= c->opts.maxit || hn == 0.0) {
        done = true;
        break;
      }
    }
    // y = H^-1 g (upper triangular), x += Z y
    for (int i = k_used - 1; i >= 0; --i) {
      double sacc = g[i];
      for (int k = i + 1; k < k_used; ++k) sacc -= H[(size_t)i * m + k] * y[k];
      y[i] = sacc / H[(size_t)i * m + i];
    }
    ck(cudaMemcpyAsync(hdev, y.data(), k_used * sizeof(double), cudaMemcpyHostToDevice, s), "y");
    multi_axpy(c->Z, n, k_used, hdev, 1.0, x, n, s);
    check_launch("fgmres update");
    ck(cudaStreamSynchronize(s), "sync");
    if (done) {
      *iters = it;
      return c->ratios.back() <= tol ? STOKES_OK : STOKES_ERR_MAXIT;
    }
    // restart: r = f - K x
    apply_Kop(c, x, r);
    axpby<double>(1.0, f, -1.0, r, n, s);
  }
  *iters = it;
  return STOKES_ERR_MAXIT;
}

bool tc_failed(stokes_ctx* c);

// FGMRES for nb right-hand sides in lockstep (contexts with nrhs > 1). Each item follows exactly
// the steps of run_fgmres (its own Hessenberg matrix, Givens rotations, restarts and stopping
// test); the preconditioner and K applies of one Arnoldi step run for all items at once, the
// Gram-Schmidt products and norms per item. Basis vector j holds the items one after the other:
// item k of V_j at V + j * nb * ntot + k * ntot. An item that has stopped is carried through the
// batched applies but no longer updated.
void run_fgmres_multi(stokes_ctx* c, const double* f, double tol, double* x, int* iters,
                      int* rcs) {
  const int nb = c->nb;
  const int64_t n = c->ntot, N = (int64_t)nb * n;
  cudaStream_t s = c->stream;
  const int m = c->opts.restart;
  const int ds = 16 + 2 * (m + 2);   // device scalars per item
  double* w = c->kv[0];
  double* r = c->kv[1];
  auto dsc = [&](int k) { return c->dsc + (size_t)k * ds; };
  std::vector<double> hs((size_t)nb * ds);
  auto read_all = [&]() {
    ck(cudaMemcpyAsync(hs.data(), c->dsc, hs.size() * sizeof(double), cudaMemcpyDeviceToHost, s),
       "read");
    ck(cudaStreamSynchronize(s), "sync");
  };
  auto put = [&](int k, int slot, double v) {   // one scalar to the device (pinned staging)
    c->pinned_multi[2 * k + (slot == 5 ? 0 : 1)] = v;
    ck(cudaMemcpyAsync(dsc(k) + slot, c->pinned_multi + 2 * k + (slot == 5 ? 0 : 1), sizeof(double),
                       cudaMemcpyHostToDevice, s), "scalar");
  };
  fill_zero(x, N * sizeof(double), s);
  c->ratios.clear();
  for (int k = 0; k < nb; ++k) dot<double>(f + k * n, f + k * n, n, c->partials, dsc(k) + 3, s);
  read_all();
  std::vector<double> fnorm(nb);
  std::vector<char> done(nb, 0);
  for (int k = 0; k < nb; ++k) {
    iters[k] = 0;
    rcs[k] = STOKES_OK;
    fnorm[k] = std::sqrt(hs[(size_t)k * ds + 3]);
    if (!std::isfinite(fnorm[k])) { rcs[k] = STOKES_ERR_NONFINITE; done[k] = 1; }
    else if (fnorm[k] == 0.0) done[k] = 1;
  }
  copy_async(r, f, N * sizeof(double), s);
  std::vector<std::vector<double>> H(nb, std::vector<double>((size_t)(m + 1) * m));
  std::vector<std::vector<double>> cs(nb, std::vector<double>(m)), sn(nb, std::vector<double>(m));
  std::vector<std::vector<double>> g(nb, std::vector<double>(m + 1)), y(nb, std::vector<double>(m));
  std::vector<int> k_used(nb, 0);
  std::vector<char> active(nb, 0), stop(nb, 0), bad(nb, 0);
  std::vector<std::vector<double>> cols(nb);
  std::vector<std::vector<double>> gram(nb, std::vector<double>((size_t)(m + 1) * (m + 1)));
  std::vector<double> hnv(nb, 0.0);
  auto any = [&](const std::vector<char>& v) {
    for (char e : v)
      if (e) return true;
    return false;
  };
  auto all_done = [&]() {
    for (char e : done)
      if (!e) return false;
    return true;
  };
  while (!all_done()) {
    for (int k = 0; k < nb; ++k)
      if (!done[k]) dot<double>(r + k * n, r + k * n, n, c->partials, dsc(k) + 4, s);
    read_all();
    for (int k = 0; k < nb; ++k) {
      active[k] = 0;
      stop[k] = 0;
      k_used[k] = 0;
      if (done[k]) continue;
      const double beta = std::sqrt(hs[(size_t)k * ds + 4]);
      if (!std::isfinite(beta)) { rcs[k] = STOKES_ERR_NONFINITE; done[k] = 1; continue; }
      if (beta == 0.0) { done[k] = 1; continue; }
      put(k, 5, beta);
      scale_inv_dev(dsc(k) + 5, r + k * n, c->V + k * n, n, s);
      std::fill(H[k].begin(), H[k].end(), 0.0);
      std::fill(g[k].begin(), g[k].end(), 0.0);
      g[k][0] = beta;
      active[k] = 1;
    }
    if (!any(active)) break;
    for (int j = 0; j < m && any(active); ++j) {
      double* Vj = c->V + (int64_t)j * N;
      double* Zj = c->Z + (int64_t)j * N;
      pk_apply(c, Vj, Zj, w);
      std::fill(bad.begin(), bad.end(), 0);
      arnoldi_gs(c, j, active, w, gram, cols, hnv, bad);   // writes V_{j+1} of every active item
      for (int k = 0; k < nb; ++k) {
        if (!active[k]) continue;
        const double hn = hnv[k];
        if (bad[k]) {
          rcs[k] = STOKES_ERR_NONFINITE;
          done[k] = 1;
          active[k] = 0;
          k_used[k] = 0;
          continue;
        }
        std::vector<double>& Hk = H[k];
        for (int i = 0; i <= j; ++i) Hk[(size_t)i * m + j] = cols[k][i];
        Hk[(size_t)(j + 1) * m + j] = hn;
        for (int i = 0; i < j; ++i) {
          const double t = cs[k][i] * Hk[(size_t)i * m + j] + sn[k][i] * Hk[(size_t)(i + 1) * m + j];
          Hk[(size_t)(i + 1) * m + j] =
              -sn[k][i] * Hk[(size_t)i * m + j] + cs[k][i] * Hk[(size_t)(i + 1) * m + j];
          Hk[(size_t)i * m + j] = t;
        }
        const double hjj = Hk[(size_t)j * m + j], hj1 = Hk[(size_t)(j + 1) * m + j];
        const double den = std::hypot(hjj, hj1);
        if (den == 0.0) {
          rcs[k] = STOKES_ERR_BREAKDOWN;
          done[k] = 1;
          active[k] = 0;
          k_used[k] = 0;
          continue;
        }
        cs[k][j] = hjj / den;
        sn[k][j] = hj1 / den;
        Hk[(size_t)j * m + j] = den;
        Hk[(size_t)(j + 1) * m + j] = 0.0;
        g[k][j + 1] = -sn[k][j] * g[k][j];
        g[k][j] = cs[k][j] * g[k][j];
        ++iters[k];
        k_used[k] = j + 1;
        const double ratio = std::fabs(g[k][j + 1]) / fnorm[k];
        if (k == 0) c->ratios.push_back(ratio);
        if (ratio <= tol || iters[k] >= c->opts.maxit || hn == 0.0) {
          active[k] = 0;
          stop[k] = 1;
          rcs[k] = ratio <= tol ? STOKES_OK : STOKES_ERR_MAXIT;
        }
      }
    }
    // y = H^-1 g (upper triangular), x += Z y, per item
    for (int k = 0; k < nb; ++k) {
      if (k_used[k] == 0) continue;
      const std::vector<double>& Hk = H[k];
      for (int i = k_used[k] - 1; i >= 0; --i) {
        double sacc = g[k][i];
        for (int q = i + 1; q < k_used[k]; ++q) sacc -= Hk[(size_t)i * m + q] * y[k][q];
        y[k][i] = sacc / Hk[(size_t)i * m + i];
      }
      double* hdev = dsc(k) + 8;
      ck(cudaMemcpyAsync(hdev, y[k].data(), k_used[k] * sizeof(double), cudaMemcpyHostToDevice, s),
         "y");
      multi_axpy(c->Z + k * n, N, k_used[k], hdev, 1.0, x + k * n, n, s);
      ck(cudaStreamSynchronize(s), "sync");   // y[k] is pageable host memory
    }
    check_launch("fgmres update");
    for (int k = 0; k < nb; ++k)
      if (stop[k]) done[k] = 1;
    if (all_done()) break;
    // restart: r = f - K x
    apply_Kop(c, x, r);
    for (int k = 0; k < nb; ++k)
      if (!done[k]) axpby<double>(1.0, f + k * n, -1.0, r + k * n, n, s);
  }
  ck(cudaStreamSynchronize(s), "sync");
}

// solve for every item of a context with nrhs > 1; per-item iterations, true residuals, codes
int solve_multi_impl(stokes_ctx* c, const double* rhs, double tol, double* x, int* iterations,
                     double* final_rel_res, int* codes) {
  const int nb = c->nb;
  const int64_t n = c->ntot;
  cudaStream_t s = c->stream;
  const int ds = 16 + 2 * (c->opts.restart + 2);
  std::vector<int> its(nb), rcs(nb);
  run_fgmres_multi(c, rhs, tol, x, its.data(), rcs.data());
  for (int k = 0; k < nb; ++k) {   // zero-mean pressure per item
    double* q = x + k * n + c->nvel;
    dot<double>(q, c->ones, c->npres, c->partials, c->dsc + (size_t)k * ds, s);
    axpy_dev(c->dsc + (size_t)k * ds, -1.0, c->zconst, q, c->npres, s);
  }
  double* tmp = c->kv[7];
  apply_Kop(c, x, tmp);
  for (int k = 0; k < nb; ++k) {
    axpby<double>(1.0, rhs + k * n, -1.0, tmp + k * n, n, s);
    dot<double>(tmp + k * n, tmp + k * n, n, c->partials, c->dsc + (size_t)k * ds + 1, s);
    dot<double>(rhs + k * n, rhs + k * n, n, c->partials, c->dsc + (size_t)k * ds + 2, s);
  }
  std::vector<double> hs((size_t)nb * ds);
  ck(cudaMemcpyAsync(hs.data(), c->dsc, hs.size() * sizeof(double), cudaMemcpyDeviceToHost, s),
     "read");
  ck(cudaStreamSynchronize(s), "sync");
  int rc = STOKES_OK;
  for (int k = 0; k < nb; ++k) {
    const double rr = hs[(size_t)k * ds + 1], ff = hs[(size_t)k * ds + 2];
    if (iterations) iterations[k] = its[k];
    if (final_rel_res) final_rel_res[k] = ff > 0 ? std::sqrt(rr / ff) : std::sqrt(rr);
    if (codes) codes[k] = rcs[k];
    if (rc == STOKES_OK && rcs[k] != STOKES_OK) rc = rcs[k];
  }
  if (tc_failed(c)) {
    c->err = "tensor-core pipeline wait timed out";
    return STOKES_ERR_CUDA;
  }
  if (rc == STOKES_ERR_MAXIT) c->err = "iteration cap reached";
  else if (rc == STOKES_ERR_NONFINITE) c->err = "non-finite value in the Krylov recurrence";
  else if (rc == STOKES_ERR_BREAKDOWN) c->err = "Krylov breakdown";
  return rc;
}

// the tensor-core pipeline raises this flag if one of its bounded waits ran out
bool tc_failed(stokes_ctx* c) {
  if (!c->of.tc) return false;
  int h[2] = {0, 0};
  ck(cudaMemcpyAsync(&h[0], c->of.tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "flag");
  if (c->ofq.tc)   // the pressure branch joins the main stream, so this read follows its kernels
    ck(cudaMemcpyAsync(&h[1], c->ofq.tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
       "flag");
  ck(cudaStreamSynchronize(c->stream), "flag");
  return h[0] != 0 || h[1] != 0;
}

int solve_impl(stokes_ctx* c, const double* rhs, double tol, double* x, int* iterations,
               double* final_rel_res) {
  int its = 0;
  int rc;
  if (c->opts.solver == STOKES_SOLVER_FGMRES) rc = run_fgmres(c, rhs, tol, x, &its);
  else rc = run_minres(c, rhs, tol, x, &its);
  normalize_pressure(c, x);
  const double rr = true_residual(c, rhs, x, c->kv[7]);
  if (iterations) *iterations = its;
  if (final_rel_res) *final_rel_res = rr;
  if (tc_failed(c)) {
    c->err = "tensor-core pipeline wait timed out";
    return STOKES_ERR_CUDA;
  }
  if (rc == STOKES_ERR_MAXIT) c->err = "iteration cap reached";
  else if (rc == STOKES_ERR_NONFINITE) c->err = "non-finite value in the Krylov recurrence";
  else if (rc == STOKES_ERR_NOT_SPD) c->err = "preconditioner is not positive definite";
  else if (rc == STOKES_ERR_BREAKDOWN) c->err = "Krylov breakdown";
  return rc;
}

// velocity-only entry points act on one item of a context with nrhs > 1
struct OneItem {
  Ops<double>& o;
  int nb;
  explicit OneItem(Ops<double>& ops) : o(ops), nb(ops.nb) { o.nb = 1; }
  ~OneItem() { o.nb = nb; }
};

// Setup tuner of the FP64 launch shapes: each candidate threads-per-block of the FP64 mode
// products (timed on the fast diagonalisation of the velocity block, FP64 preconditioner only)
// and of the FP64 banded passes (timed on the A apply) runs three times after one warm-up
// launch, with CUDA events on the context's stream; the fastest is kept. Every output is
// computed by one thread in a fixed order whatever the block size, so the choice changes timing
// only, never a result bit.
constexpr int kModeBlocks[] = {128, 256, 512};
constexpr int kBandBlocks[] = {128, 256, 512};
constexpr int kFdFused[] = {0, 1, 2, 4};

void set_shapes(stokes_ctx* c, const stokes_tuning& t) {
  c->of.tc_nsplit = c->ofq.tc_nsplit = t.tc_nsplit;
  c->od.mode_block = c->odq.mode_block = t.mode_block;
  c->od.band_block = c->odq.band_block = t.band_block;
  c->od.fd_fused = c->odq.fd_fused = t.fd_fused;
  const int band_block = t.band_block;
  if (c->quad) c->quad->band_block = band_block;
  // captured graphs hold the previous launch shapes
  for (auto& kv : c->minres_graphs) cudaGraphExecDestroy(kv.second);
  c->minres_graphs.clear();
  c->minres_graph_kernels.clear();
  for (auto& kv : c->pk_graphs) cudaGraphExecDestroy(kv.second);
  c->pk_graphs.clear();
  c->pk_graph_kernels.clear();
}

Dense transposed(const Dense& D) {
  Dense T(D.cols, D.rows);
  for (int i = 0; i < D.rows; ++i)
    for (int j = 0; j < D.cols; ++j) T(j, i) = D(i, j);
  return T;
}

void init_quad(stokes_ctx* c) {
  const QuadTables qt = build_quad_tables(c->n, c->p, c->c_pen);
  Arena& ar = c->arena;
  cudaStream_t s = c->stream;
  QuadOps* q = new QuadOps();
  c->quad = q;
  q->a = c->a;
  q->b = c->b;
  q->nq = qt.nq;
  q->nu = c->nu;
  q->nvc = c->nvc;
  q->nvel = c->nvel;
  q->n3 = (int64_t)qt.nq * qt.nq * qt.nq;
  q->s = s;
  q->band_block = c->od.band_block;
  // tables in band form (exact zeros outside the supports)
  q->BN = upload_band<double>(ar, to_band(qt.BN, 0.0), s);
  q->DN = upload_band<double>(ar, to_band(qt.DN, 0.0), s);
  q->BM = upload_band<double>(ar, to_band(qt.BM, 0.0), s);
  q->DM = upload_band<double>(ar, to_band(qt.DM, 0.0), s);
  q->BNt = upload_band<double>(ar, to_band(transposed(qt.BN), 0.0), s);
  q->DNt = upload_band<double>(ar, to_band(transposed(qt.DN), 0.0), s);
  q->BMt = upload_band<double>(ar, to_band(transposed(qt.BM), 0.0), s);
  q->DMt = upload_band<double>(ar, to_band(transposed(qt.DM), 0.0), s);
  q->Tf = upload_band<double>(ar, to_band(qt.Tface, 0.0), s);
  q->Mn = c->od.M;
  q->Mc = c->od.Mc;
  q->w = upload<double>(ar, qt.w, s);
  const int64_t nq = qt.nq, b = c->b;
  q->G = ar.alloc<double>((size_t)9 * q->n3);
  q->P = ar.alloc<double>((size_t)q->n3);
  for (int k = 0; k < 2; ++k) q->s1[k] = ar.alloc<double>((size_t)(nq * b * b));
  for (int k = 0; k < 3; ++k) q->s2[k] = ar.alloc<double>((size_t)(nq * nq * b));
  q->f1 = ar.alloc<double>((size_t)c->nvc);
  q->f2 = ar.alloc<double>((size_t)c->nvc);
  q->f3 = ar.alloc<double>((size_t)c->nvc);
}

void autotune(stokes_ctx* c) {
  cudaStream_t s = c->stream;
  double* x = c->kv[0];
  double* y = c->kv[1];
  fill_zero(x, (size_t)c->nb * c->ntot * sizeof(double), s);
  cudaEvent_t e0, e1;
  ck(cudaEventCreate(&e0), "event");
  ck(cudaEventCreate(&e1), "event");
  auto time3 = [&](auto&& fn) {
    fn();
    ck(cudaEventRecord(e0, s), "event");
    for (int r = 0; r < 3; ++r) fn();
    ck(cudaEventRecord(e1, s), "event");
    ck(cudaEventSynchronize(e1), "event");
    float ms = 0.f;
    ck(cudaEventElapsedTime(&ms, e0, e1), "event");
    return ms;
  };
  int best_mode = c->od.mode_block, best_band = c->od.band_block, best_fused = c->od.fd_fused;
  int best_split = c->of.tc_nsplit;
  if (reduced(c) && c->of.tc) {
    // tensor-core tile shape: the N columns of each 128-row tile in one work unit or two, timed
    // on the velocity fast diagonalisation and the pressure inverse (identical bits)
    float* xf = c->xf;
    float* yf = c->yf;
    fill_zero(xf, (size_t)c->nb * c->ntot * sizeof(float), s);
    float best = 1e30f;
    for (int ns : {1, 2}) {
      c->of.tc_nsplit = ns;
      const float t = time3([&] {
        c->of.fd_V(xf, yf);
        c->of.minv_Q(xf + c->nvel, yf + c->nvel);
      });
      // two units per tile only when clearly faster: timed alone, a small mesh can pick the
      // split by a few percent, and where many contexts share the GPU it is slower
      if (ns == 1 ? t < best : t < 0.90f * best) { best = t; best_split = ns; }
    }
    c->of.tc_nsplit = best_split;
  }
  if (!reduced(c)) {
    // FP64 fast diagonalisation: threads per block, six single-direction launches or three
    // fused ones (identical bits)
    float best = 1e30f;
    for (int fused : kFdFused) {
      c->od.fd_fused = fused;
      if (fused && !c->od.fused_fd_ok()) continue;
      for (int mb : kModeBlocks) {
        c->od.mode_block = mb;
        const float t = time3([&] { c->od.fd_V(x, y); });
        if (t < best) { best = t; best_mode = mb; best_fused = fused; }
      }
    }
  }
  c->od.mode_block = best_mode;
  c->od.fd_fused = best_fused;
  {
    OneItem one(c->od);
    float best = 1e30f;
    for (int bb : kBandBlocks) {
      c->od.band_block = bb;
      const float t = time3([&] { c->od.apply_A(x, y); });
      if (t < best) { best = t; best_band = bb; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  check_launch("autotune");
  set_shapes(c, stokes_tuning{best_mode, best_band, best_fused, best_split});
}


}  // namespace

// ============================================================================================
// C ABI
// ============================================================================================
extern "C" {

void stokes_default_opts(stokes_opts* o) {
  if (!o) return;
  o->c_pen = 14.0;
  o->schur = STOKES_SCHUR_INNER;
  o->precision = STOKES_PREC_FP64;
  o->solver = STOKES_SOLVER_MINRES;
  o->max_order = 3;
  o->max_steps = 4;
  o->maxit = 2000;
  o->restart = 60;
  o->stream = nullptr;
  o->nrhs = 1;
  o->autotune = 1;
  o->forward = STOKES_FORWARD_KRONECKER;
  o->outer = STOKES_OUTER_FP64;
}

int stokes_setup(stokes_t* out, int n_elems, int degree_p, double nu, const stokes_opts* opts) {
  g_setup_error.clear();
  if (!out) return fail(nullptr, STOKES_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n_elems < 1 || n_elems > 4096) return fail(nullptr, STOKES_ERR_ARG, "n_elems out of range");
  if (degree_p < 1 || degree_p > 12) return fail(nullptr, STOKES_ERR_ARG, "degree out of range");
  if (!(nu > 0.0) || !std::isfinite(nu)) return fail(nullptr, STOKES_ERR_ARG, "nu must be > 0");
  stokes_opts o;
  stokes_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.c_pen > 0.0)) o.c_pen = 14.0;
  if (o.max_order < 2 || o.max_steps < 0 || o.max_steps > 8 || o.maxit < 1 || o.restart < 1 ||
      o.restart > 400 || (o.schur != STOKES_SCHUR_INNER && o.schur != STOKES_SCHUR_NONE) ||
      o.precision < STOKES_PREC_FP64 || o.precision > STOKES_PREC_BF16 ||
      (o.solver != STOKES_SOLVER_MINRES && o.solver != STOKES_SOLVER_FGMRES))
    return fail(nullptr, STOKES_ERR_ARG, "invalid options");
  if (o.solver == STOKES_SOLVER_MINRES && o.precision != STOKES_PREC_FP64)
    return fail(nullptr, STOKES_ERR_ARG,
                "MINRES needs a fixed SPD preconditioner: use FP64 or the FGMRES solver");
  if (o.forward != STOKES_FORWARD_KRONECKER && o.forward != STOKES_FORWARD_QUADRATURE)
    return fail(nullptr, STOKES_ERR_ARG, "invalid forward operator");
  if (o.outer != STOKES_OUTER_PAIR && o.outer != STOKES_OUTER_FP64)
    return fail(nullptr, STOKES_ERR_ARG, "invalid outer arithmetic");
  if (o.nrhs < 1) o.nrhs = 1;
  if (o.nrhs > 1 && o.forward == STOKES_FORWARD_QUADRATURE)
    return fail(nullptr, STOKES_ERR_ARG, "the quadrature forward operator takes nrhs = 1");
  if (o.nrhs > 1024) return fail(nullptr, STOKES_ERR_ARG, "nrhs out of range");
  if (o.nrhs > 1 && (o.solver != STOKES_SOLVER_FGMRES ||
                     (o.precision != STOKES_PREC_TF32 && o.precision != STOKES_PREC_BF16)))
    return fail(nullptr, STOKES_ERR_ARG,
                "nrhs > 1 needs the tensor-core preconditioner (TF32 or BF16) and FGMRES");
  stokes_ctx* c = new (std::nothrow) stokes_ctx();
  if (!c) return fail(nullptr, STOKES_ERR_SETUP, "out of host memory");
  try {
    c->n = n_elems;
    c->p = degree_p;
    c->nu = nu;
    c->c_pen = o.c_pen;
    c->opts = o;
    c->a = n_elems + degree_p - 1;
    c->b = n_elems + degree_p;
    c->nvc = (int64_t)c->a * c->b * c->b;
    c->nvel = 3 * c->nvc;
    c->npres = (int64_t)c->b * c->b * c->b;
    c->ntot = c->nvel + c->npres;
    c->nb = o.nrhs;
    if (o.stream) {
      c->stream = (cudaStream_t)o.stream;
    } else {
      ck(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "stream");
      c->own_stream = true;
    }
    c->uv = build_univariate(n_elems, degree_p, o.c_pen);
    const Univariate& u = c->uv;
    std::vector<double> lN, lT;
    Dense UN, UT;
    int heN = 0, heT = 0;
    // every 1D matrix on the uniform open knot vector is centrosymmetric: split each generalised
    // eigenproblem into its even and odd halves (exact parity of the eigenvectors)
    if (!generalized_eigh_parity(u.K, u.M, lN, UN, &heN))
      throw SetupError{"mass matrix of the N basis is not positive definite"};
    if (!generalized_eigh_parity(u.Tc, u.Mc, lT, UT, &heT))
      throw SetupError{"pressure mass matrix is not positive definite"};
    for (double l : lT)
      if (!(l > 0.0)) throw SetupError{"T-check is not positive definite (raise C_pen)"};
    for (double l : lN)
      if (!(l > 0.0)) throw SetupError{"K is not positive definite"};
    const Band bM = to_band(u.M, 1e-15), bK = to_band(u.K, 1e-15);
    const Band bMc = to_band(u.Mc, 1e-15), bTc = to_band(u.Tc, 1e-15);
    std::vector<double> chol_lb_h, chol_inv_h;   // banded Cholesky factor of M-check (host)
    init_ops<double>(c, c->od, bM, bK, bMc, bTc, UN.v, lN, UT.v, lT);
    c->od.eo_N = heN;
    c->od.eo_T = heT;
    {
      // reciprocal eigenvalue sums of the fast diagonalisation, one per velocity entry
      std::vector<double> inv((size_t)c->nvel);
      for (int comp = 0; comp < 3; ++comp) {
        const Dims d = c->od.comp(comp);
        const std::vector<double>* l[3];
        for (int k = 0; k < 3; ++k) l[k] = k == comp ? &lN : &lT;
        size_t o = (size_t)comp * c->nvc;
        for (int i3 = 0; i3 < d.n3; ++i3)
          for (int i2 = 0; i2 < d.n2; ++i2)
            for (int i1 = 0; i1 < d.n1; ++i1)
              inv[o++] = 1.0 / (2.0 * nu * ((*l[0])[i1] + (*l[1])[i2] + (*l[2])[i3]));
      }
      c->od.invd = upload<double>(c->arena, inv, c->stream);
      // banded Cholesky factor of M-check (bandwidth p) for the FP64 pressure block
      const int b = c->b, p = degree_p, w = p + 1;
      const Dense& Mc = u.Mc;
      Dense L(b, b);
      for (int j = 0; j < b; ++j) {
        double d = Mc(j, j);
        for (int k = 0; k < j; ++k) d -= L(j, k) * L(j, k);
        if (!(d > 0.0)) throw SetupError{"pressure mass matrix is not positive definite"};
        L(j, j) = std::sqrt(d);
        for (int i = j + 1; i < b; ++i) {
          double t = Mc(i, j);
          for (int k = 0; k < j; ++k) t -= L(i, k) * L(j, k);
          L(i, j) = t / L(j, j);
        }
      }
      chol_lb_h.assign((size_t)b * w, 0.0);
      chol_inv_h.assign(b, 0.0);
      for (int i = 0; i < b; ++i) {
        chol_inv_h[i] = 1.0 / L(i, i);
        for (int k = std::max(0, i - p); k <= i; ++k)
          chol_lb_h[(size_t)i * w + (k - i + p)] = L(i, k);
      }
      c->od.chol_lb = upload<double>(c->arena, chol_lb_h, c->stream);
      c->od.chol_inv = upload<double>(c->arena, chol_inv_h, c->stream);
      c->od.chol_p = p;
    }
    const Ops<double>* odq = nullptr;
    if (!reduced(c)) {
      // FP64 preconditioner: the pressure recursion gets its own operator set and stream
      // the pressure branch is the longer chain at two or more steps: its blocks go first when
      // both branches have work ready
      int prio_lo = 0, prio_hi = 0;
      ck(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi), "priority range");
      ck(cudaStreamCreateWithPriority(&c->stream_q, cudaStreamNonBlocking, prio_hi), "stream");
      c->odq = c->od;
      c->odq.s = c->stream_q;
      alloc_workspace<double>(c, c->odq);
      odq = &c->odq;
    }
    if (!reduced(c)) init_hp<double>(c, c->hd, c->od, odq);   // the FP64 preconditioner
    if (reduced(c)) {
      init_ops<float>(c, c->of, bM, bK, bMc, bTc, UN.v, lN, UT.v, lT);
      const Ops<float>* ofq = nullptr;
      if (o.max_steps > 0) {
        // as in FP64: the pressure recursion (with the velocity solves of its Schur
        // approximation) runs on its own operator set, workspace and stream, concurrently with
        // the velocity recursion; the tensor-core plans of that set get their own buffers
        int prio_lo = 0, prio_hi = 0;
        ck(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi), "priority range");
        ck(cudaStreamCreateWithPriority(&c->stream_q, cudaStreamNonBlocking, prio_hi), "stream");
        c->ofq = c->of;
        c->ofq.s = c->stream_q;
        alloc_workspace<float>(c, c->ofq);
        ofq = &c->ofq;
      }
      if (o.precision == STOKES_PREC_TF32 || o.precision == STOKES_PREC_BF16)
        init_tc(c, UN, lN, UT, lT, o.precision == STOKES_PREC_BF16 ? kMmaBF16 : kMmaTF32);
      if (ofq && c->of.tc != c->ofq.tc)
        throw SetupError{"tensor-core plans of the two operator sets differ"};
      init_hp<float>(c, c->hf, c->of, ofq);
      c->xf = c->arena.alloc<float>((size_t)c->nb * c->ntot);
      c->yf = c->arena.alloc<float>((size_t)c->nb * c->ntot);
      init_pair(c, bM, bK, bMc, bTc);
    }
    if (c->nb > 1 && !c->of.tc)
      throw SetupError{"nrhs > 1: the tensor-core fast diagonalisation is not available for this "
                       "mesh"};
    // constant-pressure coefficients z = c (x) c (x) c
    std::vector<double> z((size_t)c->npres), one((size_t)c->npres, 1.0);
    const int b = c->b;
    for (int k = 0; k < b; ++k)
      for (int j = 0; j < b; ++j)
        for (int i = 0; i < b; ++i)
          z[(size_t)i + (size_t)b * (j + (size_t)b * k)] = u.const_M[i] * u.const_M[j] * u.const_M[k];
    c->zconst = upload<double>(c->arena, z, c->stream);
    c->ones = upload<double>(c->arena, one, c->stream);
    // dot scratch (partials and completion counter), then the Gram-Schmidt partials
    c->partials = c->arena.alloc<double>((size_t)kDotScratch +
                                         (size_t)kMultiDotBlocks * (2 * o.restart + 4));
    fill_zero(c->partials, kDotScratch * sizeof(double), c->stream);
    c->load1d = c->arena.alloc<double>(3 * (size_t)(c->b + 1));
    c->dsc = c->arena.alloc<double>((size_t)c->nb * (16 + 2 * (o.restart + 2)));
    c->st = c->arena.alloc<MinresState>(1);
    ck(cudaMallocHost(&c->st_host, sizeof(MinresState)), "pinned");
    ck(cudaMallocHost(&c->pinned, 64 * sizeof(double)), "pinned");
    ck(cudaMallocHost(&c->pinned_multi, 2 * (size_t)c->nb * sizeof(double)), "pinned");
    ck(cudaMallocHost(&c->pinned_h, (size_t)c->nb * (o.restart + 2) * sizeof(double)), "pinned");
    for (int i = 0; i < 8; ++i) c->kv[i] = c->arena.alloc<double>((size_t)c->nb * c->ntot);
    if (o.solver == STOKES_SOLVER_FGMRES) {
      c->V = c->arena.alloc<double>((size_t)(o.restart + 1) * c->nb * c->ntot);
      c->Z = c->arena.alloc<double>((size_t)o.restart * c->nb * c->ntot);
      c->pk_in = c->arena.alloc<double>((size_t)c->nb * c->ntot);
      c->pk_z = c->arena.alloc<double>((size_t)c->nb * c->ntot);
    }
    c->xi = c->arena.alloc<double>(c->ntot);
    c->ratio_dev = c->arena.alloc<double>(o.maxit);
    if (const char* e = std::getenv("STOKES_NO_GRAPHS")) c->use_graphs = e[0] == '0';
    if (o.forward == STOKES_FORWARD_QUADRATURE) init_quad(c);
    if (o.autotune) autotune(c);
    c->io_rhs = c->arena.alloc<double>(c->ntot);
    c->io_x = c->arena.alloc<double>(c->ntot);
    ck(cudaStreamSynchronize(c->stream), "setup");
  } catch (const CudaError& e) {
    std::string m = std::string(e.what) + ": " + cudaGetErrorString(e.e);
    stokes_destroy(c);
    return fail(nullptr, STOKES_ERR_CUDA, m);
  } catch (const SetupError& e) {
    std::string m = e.msg;
    stokes_destroy(c);
    return fail(nullptr, STOKES_ERR_SETUP, m);
  } catch (const std::bad_alloc&) {
    stokes_destroy(c);
    return fail(nullptr, STOKES_ERR_SETUP, "out of host memory");
  }
  *out = c;
  return STOKES_OK;
}

int stokes_sizes(stokes_t c, int64_t* n_vel, int64_t* n_pres) {
  if (!c) return STOKES_ERR_ARG;
  if (n_vel) *n_vel = c->nvel;
  if (n_pres) *n_pres = c->npres;
  return STOKES_OK;
}

int stokes_set_preconditioner(stokes_t c, int order, int steps) {
  if (!c) return STOKES_ERR_ARG;
  if (order < 2 || order > c->opts.max_order || steps < 0 || steps > c->opts.max_steps)
    return fail(c, STOKES_ERR_ARG, "order/steps outside [2, max_order] x [0, max_steps]");
  c->order = order;
  c->steps = steps;
  return STOKES_OK;
}

int stokes_apply_A(stokes_t c, const double* x, double* y) {
  if (!c || !x || !y) return c ? fail(c, STOKES_ERR_ARG, "null vector") : STOKES_ERR_ARG;
  try {
    OneItem one(c->od);
    c->od.apply_A(x, y);
    check_launch("apply_A");
  } catch (const CudaError& e) {
    return cuda_fail(c, e);
  }
  return STOKES_OK;
}

int stokes_apply_K(stokes_t c, const double* x, double* y) {
  if (!c || !x || !y) return c ? fail(c, STOKES_ERR_ARG, "null vector") : STOKES_ERR_ARG;
  try {
    apply_Kop(c, x, y);
    check_launch("apply_K");
  } catch (const CudaError& e) {
    return cuda_fail(c, e);
  }
  return STOKES_OK;
}

int stokes_apply_K_f32(stokes_t c, const float* x, double* y) {
  if (!c || !x || !y) return c ? fail(c, STOKES_ERR_ARG, "null vector") : STOKES_ERR_ARG;
  if (!reduced(c)) return fail(c, STOKES_ERR_ARG, "stokes_apply_K_f32 needs a reduced-precision context");
  try {
    if (c->pk.on) {
      pair_apply_K(c, x, y);
    } else {
      to_double(x, y, (int64_t)c->nb * c->ntot, c->stream);
      double* t = c->kv[1];
      apply_Kop(c, y, t);
      copy_async(y, t, (size_t)c->nb * c->ntot * sizeof(double), c->stream);
    }
    check_launch("apply_K_f32");
  } catch (const CudaError& e) {
    return cuda_fail(c, e);
  }
  return STOKES_OK;
}

int stokes_apply_hyperpower(stokes_t c, int order, int steps, const double* x, double* y) {
  if (!c || !x || !y) return c ? fail(c, STOKES_ERR_ARG, "null vector") : STOKES_ERR_ARG;
  if (order < 2 || order > c->opts.max_order || steps < 0 || steps > c->opts.max_steps)
    return fail(c, STOKES_ERR_ARG, "order/steps outside [2, max_order] x [0, max_steps]");
  try {
    apply_prec(c, order, steps, x, y);
    check_launch("apply_hyperpower");
    if (tc_failed(c)) return fail(c, STOKES_ERR_CUDA, "tensor-core pipeline wait timed out");
  } catch (const CudaError& e) {
    return cuda_fail(c, e);
  }
  return STOKES_OK;
}

int stokes_apply_P(stokes_t c, const double* x, double* y) {
  return stokes_apply_hyperpower(c, 2, 0, x, y);
}

int stokes_rhs_cavity(stokes_t c, double lid_speed, double* f) {
  if (!c || !f) return c ? fail(c, STOKES_ERR_ARG, "null vector") : STOKES_ERR_ARG;
  if (!std::isfinite(lid_speed)) return fail(c, STOKES_ERR_ARG, "lid speed must be finite");
  // Nitsche load of g = (U, 0, 0) on x2 = 1 (derived from sigma of Sec. 3.1 with boundary data):
  // f1[i1, i2, i3] = nu U (2 alpha M_i2(1) - M'_i2(1)) int N_i1 int M_i3, int M = 1.
  const Univariate& u = c->uv;
  const double alpha = c->c_pen / u.h;
  std::vector<double> f1((size_t)c->nvc);
  for (int i3 = 0; i3 < c->b; ++i3)
    for (int i2 = 0; i2 < c->b; ++i2) {
      const double g2 = c->nu * lid_speed * (2.0 * alpha * u.M_at_1[i2] - u.dM_at_1[i2]);
      for (int i1 = 0; i1 < c->a; ++i1)
        f1[(size_t)i1 + (size_t)c->a * (i2 + (size_t)c->b * i3)] = g2 * u.int_N[i1];
    }
  try {
    fill_zero(f, c->ntot * sizeof(double), c->stream);
    ck(cudaMemcpyAsync(f, f1.data(), f1.size() * sizeof(double), cudaMemcpyHostToDevice,
                       c->stream), "rhs upload");
    ck(cudaStreamSynchronize(c->stream), "rhs");
  } catch (const CudaError& e) {
    return cuda_fail(c, e);
  }
  return STOKES_OK;
}

int stokes_rhs_body(stokes_t c, int n_modes, const double* coef, const int* waves, int accumulate,
                    double* f) {
  if (!c || !f || n_modes < 0 || (n_modes > 0 && (!coef || !waves)))
    return c ? fail(c, STOKES_ERR_ARG, "invalid body-force arguments") : STOKES_ERR_ARG;
  for (int i = 0; i < 9 * n_modes; ++i)
    if (waves[i] < 1 || waves[i] > 64) return fail(c, STOKES_ERR_ARG, "wave numbers in [1, 64]");
  const Univariate& u = c->uv;
  try {
    // each mode's load is separable: its three 1D sine loads are formed on the host and their
    // outer product is accumulated on the device (modes with a zero coefficient are skipped)
    double* tmp = c->kv[7];
    fill_zero(tmp, c->nvel * sizeof(double), c->stream);
    const int ld = c->b + 1;
    std::vector<double> l(3 * (size_t)ld);
    for (int comp = 0; comp < 3; ++comp) {
      const int e1 = comp == 0 ? c->a : c->b, e2 = comp == 1 ? c->a : c->b;
      const int e3 = comp == 2 ? c->a : c->b;
      for (int m = 0; m < n_modes; ++m) {
        const double cf = coef[comp * n_modes + m];
        if (cf == 0.0) continue;
        const int* k = waves + (size_t)(comp * n_modes + m) * 3;
        const std::vector<double> l1 = comp == 0 ? sine_load_N(u, k[0]) : sine_load_M(u, k[0]);
        const std::vector<double> l2 = comp == 1 ? sine_load_N(u, k[1]) : sine_load_M(u, k[1]);
        const std::vector<double> l3 = comp == 2 ? sine_load_N(u, k[2]) : sine_load_M(u, k[2]);
        std::copy(l1.begin(), l1.end(), l.begin());
        std::copy(l2.begin(), l2.end(), l.begin() + ld);
        std::copy(l3.begin(), l3.end(), l.begin() + 2 * ld);
        // pageable source: the call returns once the host buffer has been read
        ck(cudaMemcpyAsync(c->load1d, l.data(), l.size() * sizeof(double), cudaMemcpyHostToDevice,
                           c->stream), "load upload");
        outer3_acc(c->load1d, c->load1d + ld, c->load1d + 2 * ld, cf, tmp + comp * c->nvc, e1, e2,
                   e3, c->stream);
      }
    }
    if (accumulate) {
      axpby<double>(1.0, tmp, 1.0, f, c->nvel, c->stream);
    } else {
      fill_zero(f, c->ntot * sizeof(double), c->stream);
      copy_async(f, tmp, c->nvel * sizeof(double), c->stream);
    }
    check_launch("rhs_body");
    ck(cudaStreamSynchronize(c->stream), "rhs");
  } catch (const CudaError& e) {
    return cuda_fail(c, e);
  }
  return STOKES_OK;
}

int stokes_rhs_lid_profile(stokes_t c, int ncoef, const double* theta, int accumulate,
                           double* f) {
  if (!c || !f || !theta || ncoef < 4 || ncoef > 4096)
    return c ? fail(c, STOKES_ERR_ARG, "invalid lid-profile arguments") : STOKES_ERR_ARG;
  // Nitsche load of g = (sum_k theta_k S_k(x1), 0, 0) on x2 = 1:
  // f1[i1, i2, i3] = nu (2 alpha M_i2(1) - M'_i2(1)) (int g N_i1) (int M_i3), int M = 1.
  const Univariate& u = c->uv;
  const Dense G = lid_profile_matrix(u, ncoef);
  std::vector<double> P((size_t)c->a, 0.0);
  for (int i = 0; i < c->a; ++i)
    for (int k = 0; k < ncoef; ++k) P[i] += G(i, k) * theta[k];
  const double alpha = c->c_pen / u.h;
  try {
    // rank one: f1 = P (x) g2 (x) 1, its outer product formed on the device
    const int ld = c->b + 1;
    std::vector<double> l(3 * (size_t)ld, 0.0);
    for (int i1 = 0; i1 < c->a; ++i1) l[i1] = P[i1];
    for (int i2 = 0; i2 < c->b; ++i2)
      l[ld + i2] = c->nu * (2.0 * alpha * u.M_at_1[i2] - u.dM_at_1[i2]);
    for (int i3 = 0; i3 < c->b; ++i3) l[2 * ld + i3] = 1.0;
    double* tmp = c->kv[7];
    fill_zero(tmp, c->nvc * sizeof(double), c->stream);
    ck(cudaMemcpyAsync(c->load1d, l.data(), l.size() * sizeof(double), cudaMemcpyHostToDevice,
                       c->stream), "load upload");
    outer3_acc(c->load1d, c->load1d + ld, c->load1d + 2 * ld, 1.0, tmp, c->a, c->b, c->b,
               c->stream);
    if (accumulate) {
      axpby<double>(1.0, tmp, 1.0, f, c->nvc, c->stream);
    } else {
      fill_zero(f, c->ntot * sizeof(double), c->stream);
      copy_async(f, tmp, c->nvc * sizeof(double), c->stream);
    }
    check_launch("rhs_lid_profile");
    ck(cudaStreamSynchronize(c->stream), "rhs");
  } catch (const CudaError& e) {
    return cuda_fail(c, e);
  }
  return STOKES_OK;
}

// factors of separable loads packed [m][3][ld]; chunks of terms go through the scratch vector
// kv[7] (factors, then results) and the Gram-Schmidt partials, as many as both hold
namespace {
int sep_dots_chunked(stokes_t c, const std::vector<double>& fac, int ld, int nm, const double* x,
                     int e1, int e2, int e3, double* out) {
  const int64_t fit = c->ntot / (3 * (int64_t)ld + 1);
  const int chunk = (int)std::min<int64_t>(fit, std::min(32, c->opts.restart + 2));
  if (chunk < 1) return fail(c, STOKES_ERR_ARG, "mesh too small for the load scratch");
  double* fdev = c->kv[7];
  for (int m0 = 0; m0 < nm; m0 += chunk) {
    const int k = std::min(chunk, nm - m0);
    double* rdev = fdev + (int64_t)k * 3 * ld;
    ck(cudaMemcpyAsync(fdev, fac.data() + (size_t)m0 * 3 * ld, (size_t)k * 3 * ld * sizeof(double),
                       cudaMemcpyHostToDevice, c->stream), "load factors");
    sep_dots(x, fdev, ld, k, e1, e2, e3, c->partials + kDotScratch, rdev, c->stream);
    ck(cudaMemcpyAsync(out + m0, rdev, k * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
       "dots");
    ck(cudaStreamSynchronize(c->stream), "dots");
  }
  return STOKES_OK;
}
}  // namespace

int stokes_body_load_dots(stokes_t c, int n_modes, const int* waves, const double* x,
                          double* out) {
  if (!c || !x || !out || n_modes < 1 || !waves)
    return c ? fail(c, STOKES_ERR_ARG, "invalid body-load arguments") : STOKES_ERR_ARG;
  for (int i = 0; i < 9 * n_modes; ++i)
    if (waves[i] < 1 || waves[i] > 64) return fail(c, STOKES_ERR_ARG, "wave numbers in [1, 64]");
  const Univariate& u = c->uv;
  const int ld = c->b + 1;
  try {
    for (int comp = 0; comp < 3; ++comp) {
      const int e1 = comp == 0 ? c->a : c->b, e2 = comp == 1 ? c->a : c->b;
      const int e3 = comp == 2 ? c->a : c->b;
      std::vector<double> fac((size_t)n_modes * 3 * ld, 0.0);
      for (int m = 0; m < n_modes; ++m) {
        const int* k = waves + (size_t)(comp * n_modes + m) * 3;
        const std::vector<double> l1 = comp == 0 ? sine_load_N(u, k[0]) : sine_load_M(u, k[0]);
        const std::vector<double> l2 = comp == 1 ? sine_load_N(u, k[1]) : sine_load_M(u, k[1]);
        const std::vector<double> l3 = comp == 2 ? sine_load_N(u, k[2]) : sine_load_M(u, k[2]);
        double* f = fac.data() + (size_t)m * 3 * ld;
        std::copy(l1.begin(), l1.end(), f);
        std::copy(l2.begin(), l2.end(), f + ld);
        std::copy(l3.begin(), l3.end(), f + 2 * ld);
      }
      const int rc = sep_dots_chunked(c, fac, ld, n_modes, x + comp * c->nvc, e1, e2, e3,
                                      out + comp * n_modes);
      if (rc != STOKES_OK) return rc;
    }
    check_launch("body_load_dots");
  } catch (const CudaError& e) {
    return cuda_fail(c, e);
  }
  return STOKES_OK;
}

int stokes_lid_profile_dots(stokes_t c, int ncoef, const double* x, double* out) {
  if (!c || !x || !out || ncoef < 4 || ncoef > 4096)
    return c ? fail(c, STOKES_ERR_ARG, "invalid lid-profile arguments") : STOKES_ERR_ARG;
  const Univariate& u = c->uv;
  const Dense G = lid_profile_matrix(u, ncoef);
  const double alpha = c->c_pen / u.h;
  const int ld = c->b + 1;
  std::vector<double> fac((size_t)ncoef * 3 * ld, 0.0);
  for (int k = 0; k < ncoef; ++k) {
    double* f = fac.data() + (size_t)k * 3 * ld;
    for (int i1 = 0; i1 < c->a; ++i1) f[i1] = G(i1, k);
    for (int i2 = 0; i2 < c->b; ++i2)
      f[ld + i2] = c->nu * (2.0 * alpha * u.M_at_1[i2] - u.dM_at_1[i2]);
    for (int i3 = 0; i3 < c->b; ++i3) f[2 * ld + i3] = 1.0;
  }
  try {
    const int rc = sep_dots_chunked(c, fac, ld, ncoef, x, c->a, c->b, c->b, out);
    if (rc != STOKES_OK) return rc;
    check_launch("lid_profile_dots");
  } catch (const CudaError& e) {
    return cuda_fail(c, e);
  }
  return STOKES_OK;
}

int stokes_apply_mass(stokes_t c, const double* x, double* y) {
  if (!c || !x || !y) return c ? fail(c, STOKES_ERR_ARG, "null vector") : STOKES_ERR_ARG;
  try {
    OneItem one(c->od);
    c->od.mass_V(x, y);
    check_launch("apply_mass");
  } catch (const CudaError& e) {
    return cuda_fail(c, e);
  }
  return STOKES_OK;
}

int stokes_dot(stokes_t c, const double* x, const double* y, int64_t n, double* result) {
  if (!c || !x || !y || !result || n < 0)
    return c ? fail(c, STOKES_ERR_ARG, "invalid dot arguments") : STOKES_ERR_ARG;
  try {
    dot<double>(x, y, n, c->partials, c->dsc + 12, c->stream);
    *result = read_scalar(c, c->dsc + 12);
  } catch (const CudaError& e) {
    return cuda_fail(c, e);
  }
  return STOKES_OK;
}

int stokes_solve(stokes_t c, const double* rhs, double tol, double* x, int* iterations,
                 double* final_rel_res) {
  if (!c || !rhs || !x) return c ? fail(c, STOKES_ERR_ARG, "null vector") : STOKES_ERR_ARG;
  if (!(tol > 0.0) || !(tol < 1.0)) return fail(c, STOKES_ERR_ARG, "tol must be in (0, 1)");
  if (rhs == x) return fail(c, STOKES_ERR_ARG, "rhs and x must not alias");
  try {
    if (c->nb > 1) {   // all items; the largest iteration count and residual
      std::vector<int> its(c->nb);
      std::vector<double> rr(c->nb);
      const int rc = solve_multi_impl(c, rhs, tol, x, its.data(), rr.data(), nullptr);
      if (iterations) *iterations = *std::max_element(its.begin(), its.end());
      if (final_rel_res) *final_rel_res = *std::max_element(rr.begin(), rr.end());
      return rc;
    }
    return solve_impl(c, rhs, tol, x, iterations, final_rel_res);
  } catch (const CudaError& e) {
    return cuda_fail(c, e);
  }
}

int stokes_solve_multi(stokes_t c, const double* rhs, double tol, double* x, int* iterations,
                       double* final_rel_res, int* status) {
  if (!c || !rhs || !x) return c ? fail(c, STOKES_ERR_ARG, "null vector") : STOKES_ERR_ARG;
  if (!(tol > 0.0) || !(tol < 1.0)) return fail(c, STOKES_ERR_ARG, "tol must be in (0, 1)");
  if (rhs == x) return fail(c, STOKES_ERR_ARG, "rhs and x must not alias");
  try {
    if (c->nb == 1) {
      const int rc = solve_impl(c, rhs, tol, x, iterations, final_rel_res);
      if (status) status[0] = rc;
      return rc;
    }
    return solve_multi_impl(c, rhs, tol, x, iterations, final_rel_res, status);
  } catch (const CudaError& e) {
    return cuda_fail(c, e);
  }
}

int stokes_solve_host(stokes_t c, const double* rhs_host, double tol, double* x_host,
                      int* iterations, double* final_rel_res) {
  if (!c || !rhs_host || !x_host)
    return c ? fail(c, STOKES_ERR_ARG, "null vector") : STOKES_ERR_ARG;
  if (!(tol > 0.0) || !(tol < 1.0)) return fail(c, STOKES_ERR_ARG, "tol must be in (0, 1)");
  if (c->nb > 1) return fail(c, STOKES_ERR_ARG, "stokes_solve_host takes contexts with nrhs = 1");
  try {
    const size_t bytes = c->ntot * sizeof(double);
    ck(cudaMemcpyAsync(c->io_rhs, rhs_host, bytes, cudaMemcpyHostToDevice, c->stream), "h2d");
    const int rc = solve_impl(c, c->io_rhs, tol, c->io_x, iterations, final_rel_res);
    ck(cudaMemcpyAsync(x_host, c->io_x, bytes, cudaMemcpyDeviceToHost, c->stream), "d2h");
    ck(cudaStreamSynchronize(c->stream), "d2h");
    return rc;
  } catch (const CudaError& e) {
    return cuda_fail(c, e);
  }
}

int stokes_solve_batch(stokes_t* ctxs, int count, const double* const* rhs, double tol,
                       double* const* x, int* iterations, double* final_rel_res, int* status) {
  if (!ctxs || !rhs || !x || count < 0) return STOKES_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i] || !rhs[i] || !x[i]) return STOKES_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(ctxs[i], STOKES_ERR_ARG, "contexts must be distinct");
  }
  std::vector<int> st(count, STOKES_OK);
  for (int i = 0; i < count; ++i) ctxs[i]->no_capture = true;
  std::vector<std::thread> workers;
  workers.reserve(count);
  for (int i = 0; i < count; ++i)
    workers.emplace_back([&, i] {
      st[i] = stokes_solve(ctxs[i], rhs[i], tol, x[i], iterations ? iterations + i : nullptr,
                           final_rel_res ? final_rel_res + i : nullptr);
    });
  for (auto& w : workers) w.join();
  for (int i = 0; i < count; ++i) ctxs[i]->no_capture = false;
  int rc = STOKES_OK;
  for (int i = 0; i < count; ++i) {
    if (status) status[i] = st[i];
    if (rc == STOKES_OK) rc = st[i];
  }
  return rc;
}

int stokes_last_ratios(stokes_t c, double* ratios, int capacity) {
  if (!c || (!ratios && capacity > 0) || capacity < 0) return STOKES_ERR_ARG;
  const int k = std::min<int>(capacity, (int)c->ratios.size());
  for (int i = 0; i < k; ++i) ratios[i] = c->ratios[i];
  return k;
}

int stokes_profile_begin(stokes_t c) {
  if (!c) return STOKES_ERR_ARG;
  if (!c->prof) c->prof = profiler_create();
  profiler_activate(c->prof);
  c->prof_on = true;
  c->hd.serial = true;   // per-launch event timing: no concurrent branches
  c->hf.serial = true;
  return STOKES_OK;
}

int stokes_profile_end(stokes_t c, stokes_kernel_stat* out, int capacity) {
  if (!c || !c->prof || (!out && capacity > 0) || capacity < 0) return STOKES_ERR_ARG;
  int64_t l[kNumClasses];
  double ms[kNumClasses], fl[kNumClasses], by[kNumClasses];
  profiler_collect(c->prof, l, ms, fl, by);
  profiler_activate(nullptr);
  c->prof_on = false;
  c->hd.serial = false;
  c->hf.serial = false;
  const int k = std::min(capacity, (int)kNumClasses);
  for (int i = 0; i < k; ++i) {
    out[i].kernel_class = i;
    out[i].launches = l[i];
    out[i].ms = ms[i];
    out[i].flops = fl[i];
    out[i].bytes = by[i];
  }
  return k;
}

int64_t stokes_kernel_launches(void) { return launch_count(); }

int stokes_get_tuning(stokes_t c, stokes_tuning* out) {
  if (!c || !out) return c ? fail(c, STOKES_ERR_ARG, "null tuning") : STOKES_ERR_ARG;
  out->mode_block = c->od.mode_block;
  out->band_block = c->od.band_block;
  out->fd_fused = c->od.fd_fused;
  out->tc_nsplit = c->of.tc_nsplit;
  return STOKES_OK;
}

int stokes_set_tuning(stokes_t c, const stokes_tuning* t) {
  if (!c || !t) return c ? fail(c, STOKES_ERR_ARG, "null tuning") : STOKES_ERR_ARG;
  bool ok_m = false, ok_b = false, ok_f = false;
  for (int v : kModeBlocks) ok_m = ok_m || v == t->mode_block;
  for (int v : kBandBlocks) ok_b = ok_b || v == t->band_block;
  for (int v : kFdFused) ok_f = ok_f || v == t->fd_fused;
  if (!ok_m || !ok_b) return fail(c, STOKES_ERR_ARG, "launch shape not among the candidates");
  if (!ok_f) return fail(c, STOKES_ERR_ARG, "fd_fused must be 0, 1, 2 or 4");
  if (t->tc_nsplit != 1 && t->tc_nsplit != 2)
    return fail(c, STOKES_ERR_ARG, "tc_nsplit must be 1 or 2");
  if (t->fd_fused) {
    const int keep = c->od.fd_fused;
    c->od.fd_fused = t->fd_fused;
    const bool ok = c->od.fused_fd_ok();
    c->od.fd_fused = keep;
    if (!ok) return fail(c, STOKES_ERR_ARG, "fused fast diagonalisation does not fit this mesh");
  }
  set_shapes(c, *t);
  return STOKES_OK;
}

int stokes_set_wait_limit(stokes_t c, int64_t polls) {
  if (!c) return STOKES_ERR_ARG;
  if (polls < 0 || polls > (int64_t)UINT32_MAX)
    return fail(c, STOKES_ERR_ARG, "wait limit outside [0, 2^32)");
  c->of.tc_spin = (uint32_t)polls;
  c->ofq.tc_spin = (uint32_t)polls;
  return STOKES_OK;
}

void stokes_destroy(stokes_t c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->prof) profiler_destroy(c->prof);
  if (c->st_host) cudaFreeHost(c->st_host);
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->pinned_multi) cudaFreeHost(c->pinned_multi);
  if (c->pinned_h) cudaFreeHost(c->pinned_h);
  if (c->stream_q) cudaStreamSynchronize(c->stream_q);
  cudaStream_t s = c->own_stream ? c->stream : nullptr;
  cudaStream_t sq = c->stream_q;
  delete c;   // frees the arena
  if (s) cudaStreamDestroy(s);
  if (sq) cudaStreamDestroy(sq);
}

const char* stokes_last_error(stokes_t c) {
  return c ? c->err.c_str() : g_setup_error.c_str();
}

}  // extern "C"
