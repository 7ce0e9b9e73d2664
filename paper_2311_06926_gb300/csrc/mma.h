// Tensor-core rotating mode products (k_mma.cu).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace shp {

enum { kMmaTF32 = 0, kMmaBF16 = 1 };

struct RmpArgs {
  int R;            // rows (product of the two non-contracted extents)
  int K;            // contracted extent
  int m;            // output extent along the contracted direction
  int npad;         // m rounded up to 16 (MMA N)
  int e2, e3;       // the two non-contracted extents (r = j2 + e2 j3)
  int ldy;          // output row pitch (elements) of the rotated output Y[j2 + ldy (j3 + e3 i)]
  uint32_t idesc;   // tcgen05 instruction descriptor
  float scale;      // eigenvalue scaling: divide by scale (lam_j2 + lam_j3 + lam_i) if lam_i
  const float* lam_j2;
  const float* lam_j3;
  const float* lam_i;
  float post;       // otherwise multiply by post
  void* Y;
  int nb;           // items (<= 1: one): the input holds nb * R rows, item k's rows after item
                    // k - 1's; item k's output starts ybs elements after item k - 1's
  int64_t ybs;
  int round_tf32;   // FP32 output that the next TF32 product reads: round it to TF32 (nearest)
};

struct RmpPlan {
  alignas(64) uint8_t map_x[128];    // CUtensorMap of the input rows
  alignas(64) uint8_t map_op[128];   // CUtensorMap of the padded operator
  int kind;
  bool out_bf16;
  RmpArgs args;
};

// Up to kMaxRmpJobs independent rotating products (e.g. the three velocity components) in one
// persistent launch; every plan must have the same kind and output type.
constexpr int kMaxRmpJobs = 4;

int rmp_smem_bytes(int kind, int K, int npad);
bool rmp_supported(int kind, int K, int m);
bool make_map(void* map, const void* base, int kind, int cols, int64_t rows, int ld, int box_rows);
uint32_t rmp_idesc(int kind, int npad);
// spin_limit: polls of each pipeline wait before it gives up and raises *err (0: the default,
// 2^22 polls of at least 128 ns each after the first 64); the kernel's final waits for its own
// copies and tensor-core operations in flight always use the default.
// nsplit: 1, or 2 to split every 128-row tile's N columns into two work units (two CTAs may then
// share a tile; more units for launches with few tiles). Each output column takes the same
// tensor-core operations either way, so the results are bit-identical.
void launch_rmp(const RmpPlan& p, int* err, int sms, cudaStream_t s, uint32_t spin_limit = 0,
                int nsplit = 1);
void launch_rmp_multi(const RmpPlan* const* plans, int njobs, int* err, int sms, cudaStream_t s,
                      uint32_t spin_limit = 0, int nsplit = 1);

// Copy a canonical float tensor (rows of e1 entries, R rows) into rows of pitch ld, converting
// to bfloat16 if to_bf16. nb items: item k's tensor starts xbs elements after item k - 1's in x,
// its rows follow item k - 1's in y.
void pad_rows(const float* x, int e1, int64_t R, int ld, void* y, bool to_bf16, cudaStream_t s,
              int nb = 1, int64_t xbs = 0);

}  // namespace shp
