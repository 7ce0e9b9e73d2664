// Tensor-core (tcgen05 / TMEM / TMA) mode products for the reduced-precision fast
// diagonalisation (App. A.4).
//
// Rotating mode product. A tensor with extents (e1, e2, e3), e1 fastest and its rows padded to a
// 16-byte multiple (ld >= e1), is contracted along e1 with a dense operator Op (m x e1):
//   D[r, i] = sum_j X[r][j] Op[i][j],   r = j2 + e2 j3 in [0, e2 e3),
// and written with the axes rotated, Y[j2 + ldy (j3 + e3 i)], so that the next contraction is
// again along the contiguous axis. Three rotations restore the original axis order, so the six
// products of a fast diagonalisation (U1^T, U2^T, U3^T, scale, U3, U2, U1) need no transposes.
//
// GEMM mapping on the fifth-generation tensor cores: M = 128 rows r per tile (TMEM lanes),
// N = m padded to 16 (TMEM columns, FP32 accumulator), K = e1 in 128-byte chunks. Both operands
// are K-major with the 128-byte swizzle. Op stays resident in shared memory; row tiles of X
// stream through a ring of chunk stages filled by TMA (cp.async.bulk.tensor). One elected thread
// issues tcgen05.mma; four epilogue warps read the accumulator with tcgen05.ld, apply the optional
// eigenvalue scaling and store coalesced rows. Two TMEM accumulators let the epilogue of one tile
// overlap the MMAs of the next. Every wait on an mbarrier is bounded: on timeout the kernel sets an
// error flag, stops issuing work, waits (bounded) for the tensor-core work it has issued, frees
// its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <cstring>

#include "internal.h"
#include "mma.h"
#include "profile.h"

namespace shp {
namespace {

constexpr int kTileM = 128;
constexpr int kStages = 4;
constexpr int kChunkBytes = 128;                  // one 128-byte swizzle atom of K per row
constexpr int kStageBytes = kTileM * kChunkBytes; // 16 KiB
constexpr int kEpiWarps = 8;                      // two per TMEM lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;     // warp 0 TMA, warp 1 MMA + TMEM, the rest epilogue
constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity. Returns false (and raises the shared abort
// flag and the global error flag) if it does not complete within the limit or if another role
// has already aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          int* err, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (i > 64) __nanosleep(128);
  }
  *abort_flag = 1;
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with the 128-byte swizzle: rows of 128 bytes,
// 8-row core groups 1024 bytes apart (stride byte offset), descriptor version 1, layout code 2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);        // start address
  d |= (uint64_t)1 << 16;                         // leading byte offset (unused for SW128 K-major)
  d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset
  d |= (uint64_t)1 << 46;                         // descriptor version
  d |= (uint64_t)2 << 61;                         // 128-byte swizzle
  return d;
}

template <int KIND>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                     uint32_t accumulate) {
  if (KIND == kMmaTF32) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  }
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Round to the nearest TF32 value (10 explicit mantissa bits, ties away from zero), kept in FP32
// format. The tensor cores read an FP32 operand as TF32 by dropping its low 13 mantissa bits
// (truncation, a bias toward zero of up to one TF32 ulp); operands rounded here first carry an
// unbiased error of at most half an ulp instead. Two integer operations on the bit pattern: add
// half of the dropped bits' range to the magnitude, then clear them (a carry moves into the
// exponent as it should); the host rounds the operator matrices the same way. (The conversion
// instruction with this rounding measured about 65 cycles per element in the epilogue.)
__device__ __forceinline__ float round_tf32(float v) {
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}

template <typename TO>
__device__ __forceinline__ void store_val(TO* p, float v);
template <>
__device__ __forceinline__ void store_val<float>(float* p, float v) { *p = v; }
template <>
__device__ __forceinline__ void store_val<__nv_bfloat16>(__nv_bfloat16* p, float v) {
  *p = __float2bfloat16_rn(v);
}

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct RmpJob {
  CUtensorMap map_x;
  CUtensorMap map_op;
  RmpArgs args;
  int first_tile;   // index of this job's first tile in the launch
  int ntiles;
  int nchunks;
  // N split: work unit h of a tile computes the output columns [n0[h], n0[h] + nc[h]) with the
  // operator rows of that range (nc a multiple of 16) and its own instruction descriptor
  int n0[2], nc[2];
  uint32_t idesc[2];
};

struct RmpBatch {
  RmpJob job[kMaxRmpJobs];
  int njobs;
  int total_tiles;
  int nsplit;            // work units per tile (1 or 2): the tile's N columns split in nsplit parts
  uint32_t spin_limit;   // polls of each pipeline wait before it gives up (drain waits: kSpinLimit)
};

__device__ __forceinline__ int job_of(const RmpBatch& b, int t) {
  int j = 0;
  while (j + 1 < b.njobs && t >= b.job[j + 1].first_tile) ++j;
  return j;
}

// KIND: kMmaTF32 (FP32 operands in memory) or kMmaBF16; TO: output element type. Each CTA owns a
// contiguous range of tiles over all jobs; the operator is reloaded when the range crosses into
// the next job, after the MMAs that read the previous operator have completed. Registers are
// bounded so that two CTAs fit on an SM where shared memory allows (small meshes, concurrent
// contexts): unbounded, the scaled epilogue's hoisted eigenvalues took 168 registers a thread.
template <int KIND, typename TO>
__global__ void __launch_bounds__(kThreads, 2)
    k_rmp(const __grid_constant__ RmpBatch batch, int* err) {
  // The next launch (typically the next mode product, one CTA per SM) is scheduled as SMs free
  // up; its set-up and operator copy then overlap the end of this grid.
  pdl_trigger();
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int elem = KIND == kMmaTF32 ? 4 : 2;
  const int chunk_elems = kChunkBytes / elem;
  int b_bytes = 0;
  for (int j = 0; j < batch.njobs; ++j) {
    const int bb = batch.job[j].nchunks * batch.job[j].args.npad * kChunkBytes;
    b_bytes = bb > b_bytes ? bb : b_bytes;
  }
  uint8_t* b_tile = smem;                 // operator of the current job, all K chunks
  uint8_t* a_ring = smem + b_bytes;       // kStages x 16 KiB (b_bytes is a multiple of 2 KiB)
  __shared__ uint64_t full_bar[kStages], empty_bar[kStages];
  __shared__ uint64_t b_bar, b_free_bar, drain_bar, tfull_bar[2], tempty_bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  // work units: nsplit per tile (consecutive units of one tile share its rows)
  const int ns = batch.nsplit;
  const int total_units = batch.total_tiles * ns;
  // the first total_units % gridDim.x CTAs (launched first, onto the SMs that free up first)
  // take one unit more than the others
  const int uq = total_units / (int)gridDim.x, ur = total_units - uq * (int)gridDim.x;
  const int bx = (int)blockIdx.x;
  const int u_begin = bx * uq + (bx < ur ? bx : ur);
  const int u_end = u_begin + uq + (bx < ur ? 1 : 0);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&b_bar, 1);
    mbar_init(&b_free_bar, 1);
    mbar_init(&drain_bar, 1);
    for (int t = 0; t < 2; ++t) {
      mbar_init(&tfull_bar[t], 1);
      mbar_init(&tempty_bar[t], kEpiWarps);   // one arrival per epilogue warp
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  volatile int* abort_p = &abort_flag;
  // The operators are written once at set-up, never by a preceding kernel: the first job's
  // operator copy is issued before waiting for the preceding grid, together with the barrier and
  // TMEM set-up above. Nothing else is read or written before the wait.
  int first_job = -1;
  if (warp == 0 && lane == 0 && u_begin < u_end) {
    first_job = job_of(batch, u_begin / ns);
    const RmpJob& J = batch.job[first_job];
    mbar_expect_tx(&b_bar, (uint32_t)(J.nchunks * J.args.npad * kChunkBytes));
    for (int c = 0; c < J.nchunks; ++c)
      tma_load_2d(b_tile + c * J.args.npad * kChunkBytes, &J.map_op, c * chunk_elems, 0, &b_bar);
  }
  pdl_begin();

  if (warp == 0) {
    if (lane == 0) {
      int it = 0, cur = first_job, nb = first_job >= 0 ? 1 : 0;
      bool ok = true;
      for (int u = u_begin; ok && u < u_end && !*abort_p; ++u) {
        const int t = u / ns;
        const int j = job_of(batch, t);
        const RmpJob& J = batch.job[j];
        if (j != cur) {
          // operator of job j; when replacing one, wait until its last MMAs have completed
          if (nb > 0 && !mbar_wait(&b_free_bar, (nb - 1) & 1, abort_p, err, batch.spin_limit)) break;
          mbar_expect_tx(&b_bar, (uint32_t)(J.nchunks * J.args.npad * kChunkBytes));
          for (int c = 0; c < J.nchunks; ++c)
            tma_load_2d(b_tile + c * J.args.npad * kChunkBytes, &J.map_op, c * chunk_elems, 0,
                        &b_bar);
          cur = j;
          ++nb;
        }
        const int local_tile = t - J.first_tile;
        for (int c = 0; c < J.nchunks; ++c, ++it) {
          const int s = it % kStages;
          const uint32_t ph = (it / kStages) & 1;
          if (it >= kStages && !mbar_wait(&empty_bar[s], ph ^ 1, abort_p, err, batch.spin_limit)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full_bar[s], kStageBytes);
          tma_load_2d(a_ring + s * kStageBytes, &J.map_x, c * chunk_elems, local_tile * kTileM,
                      &full_bar[s]);
        }
      }
      // bounded wait until every copy this thread issued has landed
      for (int k = (it > kStages ? it - kStages : 0); k < it; ++k) {
        const int s = k % kStages;
        for (uint32_t i = 0; i < kSpinLimit && !mbar_try_wait(&full_bar[s], (k / kStages) & 1); ++i)
          __nanosleep(128);
      }
      if (nb > 0)
        for (uint32_t i = 0; i < kSpinLimit && !mbar_try_wait(&b_bar, (nb - 1) & 1); ++i)
          __nanosleep(128);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      int it = 0, local = 0, cur = -1, nbw = 0;
      for (int u = u_begin; ok && u < u_end; ++u, ++local) {
        const int t = u / ns, h = u - t * ns;
        const int j = job_of(batch, t);
        const RmpJob& J = batch.job[j];
        if (j != cur) {
          if (!mbar_wait(&b_bar, nbw & 1, abort_p, err, batch.spin_limit)) break;
          ++nbw;
          cur = j;
        }
        const int acc = local & 1;
        const uint32_t d_tmem = tmem + acc * 256;
        if (local >= 2 && !mbar_wait(&tempty_bar[acc], ((local / 2) - 1) & 1, abort_p, err, batch.spin_limit)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int c = 0; c < J.nchunks; ++c, ++it) {
          const int s = it % kStages;
          if (!mbar_wait(&full_bar[s], (it / kStages) & 1, abort_p, err, batch.spin_limit)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a_addr = smem_u32(a_ring + s * kStageBytes);
          // the unit's operator rows start n0 rows into the chunk (n0 a multiple of 16: whole
          // 8-row swizzle atoms of 1024 bytes)
          const uint32_t b_addr =
              smem_u32(b_tile + c * J.args.npad * kChunkBytes + J.n0[h] * kChunkBytes);
#pragma unroll
          for (int k = 0; k < 4; ++k)   // 4 instructions of 32 bytes of K each
            umma<KIND>(d_tmem, sw128_desc(a_addr + 32 * k), sw128_desc(b_addr + 32 * k),
                       J.idesc[h], (c > 0 || k > 0) ? 1u : 0u);
          umma_commit(&empty_bar[s]);   // stage free once these MMAs have read it
        }
        if (!ok) break;
        umma_commit(&tfull_bar[acc]);   // accumulator ready for the epilogue
        if (u + 1 < u_end && job_of(batch, (u + 1) / ns) != j) umma_commit(&b_free_bar);
      }
      // bounded wait until every MMA this thread issued has completed
      umma_commit(&drain_bar);
      for (uint32_t i = 0; i < kSpinLimit && !mbar_try_wait(&drain_bar, 0); ++i) __nanosleep(128);
    }
  } else {
    // epilogue warps: TMEM lane quarter = warp % 4; the two warps of a quarter take alternate
    // 32-column chunks of the accumulator
    const int quarter = warp % 4;
    const int half = (warp - 2) / 4;
    const int row_in_tile = quarter * 32 + lane;
    int local = 0;
    for (int u = u_begin; u < u_end; ++u, ++local) {
      const int t = u / ns, h = u - t * ns;
      const RmpJob& J = batch.job[job_of(batch, t)];
      const RmpArgs& args = J.args;
      const int n0 = J.n0[h], nc = J.nc[h];
      const int acc = local & 1;
      int ok = 1;
      if (lane == 0) ok = mbar_wait(&tfull_bar[acc], (local / 2) & 1, abort_p, err, batch.spin_limit) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int r = (t - J.first_tile) * kTileM + row_in_tile;
      const int nbi = args.nb > 1 ? args.nb : 1;
      const bool valid = r < args.R * nbi;
      TO* yrow = reinterpret_cast<TO*>(args.Y);
      float lam_r = 0.f;
      if (valid) {
        const int k = nbi > 1 ? r / args.R : 0;   // item
        const int rr = r - k * args.R;
        const int j2 = rr % args.e2, j3 = rr / args.e2;
        yrow += (int64_t)k * args.ybs + j2 + (int64_t)args.ldy * j3;
        if (args.lam_i) lam_r = args.lam_j2[j2] + args.lam_j3[j3];
      }
      const int64_t stride_i = (int64_t)args.ldy * args.e3;
      const float post = args.post, scale = args.scale;
      const bool rt = args.round_tf32 != 0;
      for (int c0 = half * 32; c0 < nc; c0 += 64) {
        float v[32];
        tmem_ld32(tmem + acc * 256 + ((uint32_t)(quarter * 32) << 16) + c0, v);
        const int gc = n0 + c0;   // output column of the chunk's first accumulator column
        if (valid && gc < args.m) {
          const int lim = args.m - gc < nc - c0 ? args.m - gc : nc - c0;
          const int kmax = lim < 32 ? lim : 32;
          TO* yp = yrow + stride_i * gc;
          if (args.lam_i) {
            // the chunk's eigenvalues into registers before the first store: loaded between
            // the stores (which may alias them for the compiler), each waited a full load latency
            const float* li = args.lam_i + gc;
            float lk[32];
            if (kmax == 32) {
#pragma unroll
              for (int k = 0; k < 32; ++k) lk[k] = __ldg(li + k);
#pragma unroll
              for (int k = 0; k < 32; ++k) {
                const float val = __fdividef(v[k], scale * (lam_r + lk[k]));
                store_val<TO>(yp + stride_i * k, rt ? round_tf32(val) : val);
              }
            } else {
#pragma unroll
              for (int k = 0; k < 32; ++k) lk[k] = k < kmax ? __ldg(li + k) : 1.f;
#pragma unroll
              for (int k = 0; k < 32; ++k) {
                if (k < kmax) {
                  const float val = __fdividef(v[k], scale * (lam_r + lk[k]));
                  store_val<TO>(yp, rt ? round_tf32(val) : val);
                }
                yp += stride_i;
              }
            }
          } else if (kmax == 32) {
            // full chunk: no per-element predicate (it cost twice the time of the stores)
            if (rt) {
#pragma unroll
              for (int k = 0; k < 32; ++k) store_val<TO>(yp + stride_i * k, round_tf32(v[k] * post));
            } else {
#pragma unroll
              for (int k = 0; k < 32; ++k) store_val<TO>(yp + stride_i * k, v[k] * post);
            }
          } else {
#pragma unroll
            for (int k = 0; k < 32; ++k) {
              if (k < kmax) {
                const float val = v[k] * post;
                store_val<TO>(yp, rt ? round_tf32(val) : val);
              }
              yp += stride_i;
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty_bar[acc]);
    }
  }
  // drain: make sure no tensor-core work of this CTA is in flight before TMEM is freed
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

template <typename TO>
// One warp per row (rows of all items in order), lanes along the row: coalesced loads and stores,
// one division per row instead of one per element.
__global__ void k_pad_rows(const float* __restrict__ x, int e1, int64_t R, int ld,
                           TO* __restrict__ y, int nb, int64_t xbs) {
  pdl_trigger();   // the mode product that reads this copy sets up while the copy runs
  pdl_begin();
  const int64_t rows = R * nb;
  const int lane = threadIdx.x % 32;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
  for (int64_t r = w0; r < rows; r += nw) {
    const int64_t k = nb > 1 ? r / R : 0;     // item
    const float* src = x + k * xbs + (r - k * R) * e1;
    TO* dst = y + r * ld;
    for (int j = lane; j < e1; j += 32) {
      // the FP32 copy feeds TF32 products: rounded to TF32 here (BF16 rounds in store_val)
      if constexpr (sizeof(TO) == 4) store_val<TO>(dst + j, round_tf32(src[j]));
      else store_val<TO>(dst + j, src[j]);
    }
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

}  // namespace

int rmp_smem_bytes(int kind, int K, int npad) {
  const int elem = kind == kMmaTF32 ? 4 : 2;
  const int nchunks = (K + kChunkBytes / elem - 1) / (kChunkBytes / elem);
  return 1024 + nchunks * npad * kChunkBytes + kStages * kStageBytes;
}

bool rmp_supported(int kind, int K, int m) {
  const int npad = round_up(m, 16);
  return npad <= 256 && rmp_smem_bytes(kind, K, npad) <= 220 * 1024;
}

// 2D tensor map over rows of `cols` valid elements (row pitch `ld` elements, 16-byte multiple),
// box = (128 bytes of columns) x box_rows, 128-byte swizzle, zero fill out of range.
bool make_map(void* map, const void* base, int kind, int cols, int64_t rows, int ld, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const int elem = kind == kMmaTF32 ? 4 : 2;
  if (((uintptr_t)base) % 16 != 0 || ((int64_t)ld * elem) % 16 != 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * elem};
  cuuint32_t box[2] = {(cuuint32_t)(kChunkBytes / elem), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(reinterpret_cast<CUtensorMap*>(map),
                   kind == kMmaTF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                    : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                   2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

uint32_t rmp_idesc(int kind, int npad) {
  const uint32_t fmt = kind == kMmaTF32 ? 2u : 1u;   // TF32 = 2 (kind::tf32), BF16 = 1 (kind::f16)
  uint32_t d = 0;
  d |= 1u << 4;                        // accumulator format F32
  d |= fmt << 7;                       // A format
  d |= fmt << 10;                      // B format
  d |= (uint32_t)(npad >> 3) << 17;    // N
  d |= (uint32_t)(kTileM >> 4) << 24;  // M
  return d;
}

template <int KIND, typename TO>
void launch_rmp_t(const RmpPlan* const* plans, int njobs, int* err, int sms, cudaStream_t s,
                  uint32_t spin_limit, int nsplit) {
  RmpBatch b{};
  b.njobs = njobs;
  // two units per tile only when every job's N splits into two multiples of 16
  for (int j = 0; j < njobs && nsplit > 1; ++j)
    if (plans[j]->args.npad < 32) nsplit = 1;
  b.nsplit = nsplit > 1 ? 2 : 1;
  int tiles = 0, smem = 0;
  double flops = 0, bytes = 0;
  const int elem = KIND == kMmaTF32 ? 4 : 2;
  for (int j = 0; j < njobs; ++j) {
    const RmpPlan& p = *plans[j];
    RmpJob& J = b.job[j];
    std::memcpy(&J.map_x, p.map_x, sizeof(CUtensorMap));
    std::memcpy(&J.map_op, p.map_op, sizeof(CUtensorMap));
    J.args = p.args;
    J.first_tile = tiles;
    const int64_t rows = (int64_t)p.args.R * (p.args.nb > 1 ? p.args.nb : 1);
    J.ntiles = (int)((rows + kTileM - 1) / kTileM);
    J.nchunks = (p.args.K + kChunkBytes / elem - 1) / (kChunkBytes / elem);
    if (b.nsplit == 2) {
      J.nc[0] = round_up((p.args.npad + 1) / 2, 16);
      J.nc[1] = p.args.npad - J.nc[0];
    } else {
      J.nc[0] = p.args.npad;
      J.nc[1] = 0;
    }
    J.n0[0] = 0;
    J.n0[1] = J.nc[0];
    J.idesc[0] = rmp_idesc(KIND, J.nc[0]);
    J.idesc[1] = b.nsplit == 2 ? rmp_idesc(KIND, J.nc[1]) : 0u;
    tiles += J.ntiles;
    const int sm = rmp_smem_bytes(KIND, p.args.K, p.args.npad);
    smem = sm > smem ? sm : smem;
    flops += 2.0 * rows * p.args.m * p.args.K;
    bytes += (double)rows * (p.args.K * elem + p.args.m * (double)sizeof(TO));
  }
  b.total_tiles = tiles;
  b.spin_limit = spin_limit > 0 ? spin_limit : kSpinLimit;
  const int units = tiles * b.nsplit;
  const int grid = units < sms ? units : sms;
  if (smem < 116 * 1024) smem = 116 * 1024;   // one CTA, one 512-column TMEM allocation per SM
  static std::atomic<int> attr{0};
  raise_smem_limit(k_rmp<KIND, TO>, attr, 220 * 1024);
  launch_begin(kClassMma, s);
  launch_k(k_rmp<KIND, TO>, grid, kThreads, smem, s, b, err);
  launch_end(kClassMma, s, flops, bytes);
}

void launch_rmp_multi(const RmpPlan* const* plans, int njobs, int* err, int sms, cudaStream_t s,
                      uint32_t spin_limit, int nsplit) {
  const RmpPlan& p = *plans[0];
  if (p.kind == kMmaTF32)
    launch_rmp_t<kMmaTF32, float>(plans, njobs, err, sms, s, spin_limit, nsplit);
  else if (p.out_bf16)
    launch_rmp_t<kMmaBF16, __nv_bfloat16>(plans, njobs, err, sms, s, spin_limit, nsplit);
  else launch_rmp_t<kMmaBF16, float>(plans, njobs, err, sms, s, spin_limit, nsplit);
}
void launch_rmp(const RmpPlan& p, int* err, int sms, cudaStream_t s, uint32_t spin_limit,
                int nsplit) {
  const RmpPlan* one = &p;
  launch_rmp_multi(&one, 1, err, sms, s, spin_limit, nsplit);
}

void pad_rows(const float* x, int e1, int64_t R, int ld, void* y, bool to_bf16, cudaStream_t s,
              int nb, int64_t xbs) {
  if (nb < 1) nb = 1;
  const int64_t total = (int64_t)e1 * R * nb;
  int64_t blocks = (R * nb + 7) / 8;   // 8 warps (rows) per block
  if (blocks > 152 * 32) blocks = 152 * 32;
  launch_begin(kClassVector, s);
  if (to_bf16)
    launch_k(k_pad_rows<__nv_bfloat16>, (int)blocks, 256, 0, s, x, e1, R, ld,
             static_cast<__nv_bfloat16*>(y), nb, xbs);
  else
    launch_k(k_pad_rows<float>, (int)blocks, 256, 0, s, x, e1, R, ld, static_cast<float*>(y), nb,
             xbs);
  launch_end(kClassVector, s, 0.0, (double)total * (to_bf16 ? 6.0 : 8.0));
}

}  // namespace shp
