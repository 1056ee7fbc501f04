// Shared host/device definitions of the IBMI library (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/ibmi.h"

namespace ibmi {

// Thread-local text of the last CUDA error; exposed through ibmi_last_error().
void set_last_error(const std::string& s);

#define IBMI_CUDA_TRY(expr)                                                        \
  do {                                                                             \
    cudaError_t _e = (expr);                                                       \
    if (_e != cudaSuccess) {                                                       \
      ::ibmi::set_last_error(std::string(#expr) + ": " + cudaGetErrorString(_e));  \
      return _e == cudaErrorMemoryAllocation ? IBMI_ERR_OOM : IBMI_ERR_CUDA;       \
    }                                                                              \
  } while (0)

#define IBMI_TRY(expr)                      \
  do {                                      \
    ibmi_status _s = (expr);                \
    if (_s != IBMI_OK) return _s;           \
  } while (0)

// Launch accounting and per-class event timing (ibmi_prof_*).
bool prof_on();
void note_launch(int n = 1);
void prof_begin(int kclass, cudaStream_t st);
void prof_end(int kclass, cudaStream_t st, double flops, double alg_flops);

// Scoped helper: times everything launched on `st` inside the scope as class
// k.  flops: operations issued to the executing unit (a sliced product counts
// every slice product); alg: the flops of the product the method itself asks
// for (its share, for a launch that forms part of one); negative = flops.
struct ProfScope {
  int k; cudaStream_t st; double flops, alg;
  ProfScope(int k_, cudaStream_t s, double f, double a = -1.0) : k(k_), st(s), flops(f), alg(a) { prof_begin(k, st); }
  ~ProfScope() { prof_end(k, st, flops, alg < 0.0 ? flops : alg); }
};

// Logical index l in [0, n) of I^c -> physical row/column of A or H, for the
// set [lo, hi): skip the gap of width (hi - lo) starting at lo.
struct GapMap {
  int64_t at;   // first logical index that is shifted (= lo)
  int64_t len;  // shift (= hi - lo); 0 = identity map
  __host__ __device__ __forceinline__ int64_t operator()(int64_t l) const {
    return l + (l >= at ? len : 0);
  }
};

// Device-side status word shared by the kernels of one call.
struct DevStatus {
  int32_t code;       // 0 ok, else an ibmi_status
  int32_t block;      // failing set for NOT_SPD
  int64_t pivot;      // failing pivot (row inside the block)
};

}  // namespace ibmi
