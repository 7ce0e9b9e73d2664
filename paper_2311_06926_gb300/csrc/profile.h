// Launch accounting: a process-wide launch counter and an optional per-thread profiler that
// brackets each launch with CUDA events on the launching stream and records the launch's
// algorithmic flops and bytes.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace shp {

enum KernelClass {
  kClassBand = 0,      // banded Kronecker passes
  kClassMode = 1,      // dense mode products (fast diagonalisation, pressure mass inverse)
  kClassDiv = 2,       // discrete divergence and its transpose
  kClassVector = 3,    // Krylov vector kernels, dot products, conversions
  kClassMma = 4,       // tensor-core mode products
  kClassLine = 5,      // banded Cholesky line solves (FP64 pressure block)
  kClassBand64 = 6,    // FP64 banded Kronecker passes (class 0 then holds the FP32 ones)
  kClassPair = 7,      // banded passes and divergence in pair-of-FP32 arithmetic
  kNumClasses = 8
};

void launch_begin(int cls, cudaStream_t s);
void launch_end(int cls, cudaStream_t s, double flops, double bytes);
int64_t launch_count();
// Adjusts the counter by n (kernels of a captured graph: counted on replay, not on capture).
void launch_add(int64_t n);
// While set (per host thread), launches are being captured into a graph and are not counted.
void set_capturing(bool on);

struct Profiler;
Profiler* profiler_create();
void profiler_destroy(Profiler* p);
void profiler_activate(Profiler* p);   // nullptr: deactivate (this thread)
// Per class: launches, milliseconds (sum of event intervals), flops, bytes. Synchronizes.
void profiler_collect(Profiler* p, int64_t* launches, double* ms, double* flops, double* bytes);

}  // namespace shp
