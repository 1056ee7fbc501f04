// tcgen05 / TMEM split-BF16 GEMM for sm_103a (internal).
//
// C[i, j] = sum_{s + u <= S-1} sum_k A_s[i, k] * B_u[j, k]
//
// A_s (M x K) and B_u (N x K) are BF16 slices, both K-major (row-major with K
// contiguous), read by TMA in 64-wide K blocks with the 128-byte swizzle.  The
// slices of a value x are x_0 = bf16(x), x_1 = bf16(x - x_0), ... so the
// triangle of slice products reproduces x*y to about 8*S bits; S = 2 is the
// classic three-product BF16x3 scheme, S = 3 the six-product scheme.  The
// accumulator is FP32 in tensor memory (128 lanes x BN columns).
//
// The kernel is persistent: each CTA walks the 128 x BN output tiles (and K
// splits) tile = blockIdx.x, blockIdx.x + gridDim.x, ...  Roles:
//   warp 0   : one thread issues the TMA loads of each stage (S A-tiles and
//              S B-tiles) into a ring of shared-memory stages that runs on
//              across tiles;
//   warp 1   : allocates TMEM for two accumulators; one thread issues
//              tcgen05.mma into accumulator (tile & 1) and commits;
//   warps 2-5: epilogue; each drains its 32-lane quadrant of the accumulator
//              with tcgen05.ld, hands 16 FP32 values at a time to the functor
//              and frees the accumulator, so the MMAs of tile i+1 overlap the
//              epilogue of tile i.
// Every mbarrier wait is bounded (about 2 s of wall time); on expiry the
// kernel records an error code in *err and finishes without hanging.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "common.cuh"

namespace ibmi {
namespace tc {

constexpr int BM = 128;       // rows per tile (one TMEM lane per row)
constexpr int BK = 64;        // BF16 elements per K block = one 128-byte swizzle row
constexpr int THREADS = 192;  // 6 warps
constexpr int ERR_TIMEOUT = 7;

struct Maps {
  CUtensorMap a[4];
  CUtensorMap b[4];
};

struct Tiles {
  int64_t M;        // rows of C that exist (rows >= M are computed but not passed on)
  int64_t a_row0;   // TMA row of C row 0 inside the A tensor
  int64_t b_row0;   // TMA row of C column 0 inside the B tensor
  int nt0;          // N tiles of the first range: physical column tile t
  int nt1_first;    // physical column tile of logical N tile nt0
  int kt0_end;      // K tiles [0, kt0_end) then [kt1_begin, kt1_end)
  int kt1_begin;
  int kt1_end;
  int splits;       // K splits
  int* err;         // error word (0 = ok)
  int grid_n = 0;   // N tiles, M tiles (filled in by launch())
  int grid_m = 0;
  // Programmatic dependent launch: the kernel may start while the previous
  // kernel on the stream (another k_tc_gemm that set this) finishes.  Only
  // for launches whose operands no k_tc_gemm writes: the epilogue waits for
  // the previous grid before its first global access, then lets the next
  // launch begin.
  int pdl = 0;
  // Per 128-row tile K-tile ranges [x, y) (device array of grid_m entries;
  // splits == 1, kt0_end >= every y): rows of different problems stacked in
  // one launch, each with its own K range.
  const int2* mkr = nullptr;
  // Lower tiles only (square tiles, grid_n == grid_m, identity N-tile map):
  // the units are the tiles on or below the diagonal, for a symmetric result
  // whose consumer reads element (i, j) with j > i from (j, i).
  int lower = 0;
  // Self-test of the bounded waits only: the producer issues no loads, so the
  // MMA thread's first wait expires and the kernel takes its error exit.
  int starve = 0;
  // Batch of independent problems of the same shape (nb > 0): the maps are
  // 3-D with the problem index as third coordinate, the units are the units
  // of one problem for each of nb problems, problem bsel[i] (or i) for the
  // i-th block of units; the epilogue learns the problem through `bat`.
  int nb = 0;
  const int* bsel = nullptr;
};

__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Work unit -> output tile, split index and K-tile range: unit u is tile
// u mod (grid_n grid_m) of K split u / (grid_n grid_m).
struct Unit {
  int tile, z, kb, nk;
};
__host__ __device__ inline int tiles_per_split(const Tiles& t) {
  return t.lower ? t.grid_m * (t.grid_m + 1) / 2 : t.grid_n * t.grid_m;
}
__host__ __device__ inline int unit_count(const Tiles& t) { return tiles_per_split(t) * t.splits; }
__device__ __forceinline__ Unit unit_of(const Tiles& t, int u, int nk) {
  Unit r;
  r.tile = u;
  r.z = u / tiles_per_split(t);
  if (t.lower) {   // v-th lower tile: row mt with mt (mt + 1) / 2 <= v, column v - mt (mt + 1) / 2
    const int v = u - r.z * tiles_per_split(t);
    int mt = (int)((sqrtf(8.0f * (float)v + 1.0f) - 1.0f) * 0.5f);
    while ((mt + 1) * (mt + 2) / 2 <= v) ++mt;
    while (mt * (mt + 1) / 2 > v) --mt;
    r.tile = mt * t.grid_n + (v - mt * (mt + 1) / 2);   // same encoding as a full grid
  }
  if (t.mkr) {
    const int2 kr = t.mkr[(u / t.grid_n) % t.grid_m];
    r.kb = kr.x;
    r.nk = kr.y - kr.x;
    return r;
  }
  r.kb = (int)((int64_t)nk * r.z / t.splits);
  r.nk = (int)((int64_t)nk * (r.z + 1) / t.splits) - r.kb;
  return r;
}

// Unit u of a (possibly batched) launch: its problem b and its unit within the problem.
__device__ __forceinline__ Unit unit_at(const Tiles& t, int u, int nk, int& b) {
  b = 0;
  if (t.nb > 0) {
    const int per = unit_count(t);
    const int bi = u / per;
    b = t.bsel ? t.bsel[bi] : bi;
    u -= bi * per;
  }
  return unit_of(t, u, nk);
}
__host__ __device__ inline int total_units(const Tiles& t) { return unit_count(t) * (t.nb > 0 ? t.nb : 1); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the completion of phase `parity`.  Returns false (and sets
// *err) after ~2 s, or as soon as another thread has flagged an error.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* err) {
  if (mbar_try_wait(b, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(b, parity)) return true;
    if ((it & 127) == 0) {
      if (*(volatile int*)err != 0) return false;
      if (globaltimer() - t0 > 2000000000ull) {
        atomicExch(err, ERR_TIMEOUT);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(smem_u32(dst)), "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
      ::"r"(smem_u32(dst)), "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row core groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address, bits 0-13
  d |= (uint64_t)1 << 16;                      // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset, bits 32-45
  d |= (uint64_t)1 << 46;                      // descriptor version
  d |= (uint64_t)2 << 61;                      // swizzle: 128 B
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulate, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem_d), "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// Error exit of the MMA thread: commit every tcgen05.mma it has issued to the
// spare barrier `drain` (count 1, phase 0) and wait, bounded by 1 s, for its
// arrival, so that no MMA still writes the accumulators when TMEM is freed.
// (With nothing issued the commit arrives at once.)
__device__ __forceinline__ void mma_drain_on_error(uint64_t* drain) {
  mma_commit(drain);
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < 1000000000ull) {
  }
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Epilogue functors: operator()(row, col0, z, v[16]) per 16-column chunk of a
// row (called by the thread owning that TMEM lane), then done(quadrant) once.
struct EpiBase {
  int bat = 0;   // problem of the current unit (batched launches)
  __device__ __forceinline__ void done(int) {}
};
template <class E, class = void>
struct has_bat : std::false_type {};
template <class E>
struct has_bat<E, std::void_t<decltype(&E::bat)>> : std::true_type {};
// An epilogue with a member unit_end(quadrant, tile) is told when its warp has
// passed on the last chunk of a unit (per-unit reductions).
template <class E, class = void>
struct has_unit_end : std::false_type {};
template <class E>
struct has_unit_end<E, std::void_t<decltype(&E::unit_end)>> : std::true_type {};

// An epilogue with a member warp_tile(row0, j0, z, stage, lane) gets each
// warp's 32 x 16 block through shared memory (stage[r * 17 + c] = row r,
// column c) so that its global accesses can be coalesced along rows; others
// get one row per lane.
template <class E, class = void>
struct has_warp_tile : std::false_type {};
template <class E>
struct has_warp_tile<E, std::void_t<decltype(&E::warp_tile)>> : std::true_type {};
constexpr uint32_t STAGE_TILE_BYTES = 4 * 32 * 17 * 4;   // four epilogue warps

// 32 lanes x 16 columns of 32-bit: thread t of the warp gets lane (quadrant + t).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Pipeline depth: when three stages fit in half of the 227 KB of shared
// memory, two CTAs share an SM (one CTA's epilogue overlaps the other's main
// loop); otherwise one CTA per SM with as many stages as fit.
template <int S, int BN>
struct Cfg {
  static constexpr uint32_t A_BYTES = BM * BK * 2;
  static constexpr uint32_t B_BYTES = BN * BK * 2;
  static constexpr uint32_t STAGE_BYTES = S * (A_BYTES + B_BYTES);
  static constexpr bool TWO_PER_SM = 3 * STAGE_BYTES + 1280 <= 113 * 1024;
  static constexpr int STAGES =
      TWO_PER_SM ? 3 : ((200 * 1024) / STAGE_BYTES >= 4 ? 4 : (200 * 1024) / STAGE_BYTES);
  static constexpr uint32_t SMEM = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
  // two accumulators; an allocation is a power of two of at least 32 columns
  static constexpr uint32_t TMEM_COLS = 2 * BN <= 32 ? 32 : 2 * BN <= 64 ? 64 : 2 * BN <= 128 ? 128 : 2 * BN <= 256 ? 256 : 512;
  static constexpr int CTAS_PER_SM = TWO_PER_SM && 2 * TMEM_COLS <= 512 ? 2 : 1;
  static_assert(TMEM_COLS <= 512, "two accumulators must fit in TMEM");
  static_assert(STAGES >= 2, "tile too large for two stages");
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N for M = 128");
};

template <int S, int BN, class Epi>
__global__ void __launch_bounds__(THREADS, Cfg<S, BN>::CTAS_PER_SM) k_tc_gemm(const __grid_constant__ Maps maps,
                                                                             const Tiles t, Epi epi) {
  using C = Cfg<S, BN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* tiles = smem;
  uint64_t* full = (uint64_t*)(smem + C::STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + C::STAGES;
  uint64_t* accf = empty + C::STAGES;   // [2] accumulator ready
  uint64_t* acce = accf + 2;            // [2] accumulator drained
  uint64_t* drain = acce + 2;           // MMA completion on an error exit
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int units = total_units(t);
  const int nk0 = t.kt0_end;
  const int nk = t.kt0_end + (t.kt1_end - t.kt1_begin);

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 4);   // one arrival per epilogue warp
    }
    mbar_init(drain, 1);
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, C::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0 && !t.starve) {  // TMA producer
      int kc = 0;     // k blocks issued so far (ring position)
      bool ok = true;
      for (int u = blockIdx.x; ok && u < units; u += gridDim.x) {
        int bb;
        const Unit w = unit_at(t, u, nk, bb);
        const int ntl = w.tile % t.grid_n, mt = (w.tile / t.grid_n) % t.grid_m;
        const int ntp = ntl < t.nt0 ? ntl : t.nt1_first + (ntl - t.nt0);
        const int64_t n0 = (int64_t)ntp * BN;
        const int kb = w.kb, my_nk = w.nk;
        for (int it = 0; it < my_nk; ++it, ++kc) {
          const int st = kc % C::STAGES;
          const uint32_t ph = (uint32_t)(kc / C::STAGES) & 1u;
          if (!mbar_wait(&empty[st], ph ^ 1u, t.err)) { ok = false; break; }
          const int kt = kb + it;
          const int ktp = kt < nk0 ? kt : t.kt1_begin + (kt - nk0);
          const int kx = ktp * BK;
          uint8_t* sa = tiles + st * C::STAGE_BYTES;
          uint8_t* sb = sa + S * C::A_BYTES;
          mbar_expect_tx(&full[st], C::STAGE_BYTES);
          const int ya = (int)(t.a_row0 + (int64_t)mt * BM), yb = (int)(t.b_row0 + n0);
          if (t.nb > 0) {
#pragma unroll
            for (int s = 0; s < S; ++s) tma_load_3d(sa + s * C::A_BYTES, &maps.a[s], &full[st], kx, ya, bb);
#pragma unroll
            for (int s = 0; s < S; ++s) tma_load_3d(sb + s * C::B_BYTES, &maps.b[s], &full[st], kx, yb, bb);
          } else {
#pragma unroll
            for (int s = 0; s < S; ++s) tma_load_2d(sa + s * C::A_BYTES, &maps.a[s], &full[st], kx, ya);
#pragma unroll
            for (int s = 0; s < S; ++s) tma_load_2d(sb + s * C::B_BYTES, &maps.b[s], &full[st], kx, yb);
          }
        }
      }
      // On an error exit, wait (bounded) for the copies still in flight.
      if (*(volatile int*)t.err != 0) {
        for (int k = kc - C::STAGES < 0 ? 0 : kc - C::STAGES; k < kc; ++k) {
          const int st = k % C::STAGES;
          const uint32_t ph = (uint32_t)(k / C::STAGES) & 1u;
          const uint64_t t0 = globaltimer();
          while (!mbar_try_wait(&full[st], ph) && globaltimer() - t0 < 1000000000ull) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      constexpr uint32_t idesc = idesc_bf16(BM, BN);
      int kc = 0;
      int local = 0;
      bool ok = true;
      for (int u = blockIdx.x; ok && u < units; u += gridDim.x, ++local) {
        int bb;
        const int my_nk = unit_at(t, u, nk, bb).nk;
        const int buf = local & 1;
        const uint32_t use = (uint32_t)(local >> 1);
        if (!mbar_wait(&acce[buf], (use & 1u) ^ 1u, t.err)) break;   // accumulator drained
        tc_fence_after();
        const uint32_t dacc = tmem + (uint32_t)(buf * BN);
        for (int it = 0; it < my_nk; ++it, ++kc) {
          const int st = kc % C::STAGES;
          const uint32_t ph = (uint32_t)(kc / C::STAGES) & 1u;
          if (!mbar_wait(&full[st], ph, t.err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(tiles + st * C::STAGE_BYTES);
          const uint32_t sb = sa + S * C::A_BYTES;
#pragma unroll
          for (int s = 0; s < S; ++s)
#pragma unroll
            for (int u = 0; s + u < S; ++u)
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) {
                const uint64_t da = sdesc_sw128(sa + s * C::A_BYTES + kk * 32);
                const uint64_t db = sdesc_sw128(sb + u * C::B_BYTES + kk * 32);
                mma_bf16(dacc, da, db, idesc, (it | s | u | kk) != 0 ? 1u : 0u);
              }
          mma_commit(&empty[st]);
        }
        mma_commit(&accf[buf]);
      }
      if (!ok || *(volatile int*)t.err != 0) mma_drain_on_error(drain);
    }
  } else {  // epilogue warps 2..5
    const int q = warp & 3;
    const int row = q * 32 + lane;
    if (t.pdl) {
      grid_dependency_wait();   // the previous grid's writes are complete and visible
      if (warp == 2 && lane == 0) grid_launch_dependents();
    }
    Epi e = epi;
    float* stage = (float*)(smem + C::STAGES * C::STAGE_BYTES + 256) + q * 32 * 17;   // warp_tile epilogues only
    int local = 0;
    for (int u = blockIdx.x; u < units; u += gridDim.x, ++local) {
      int bb;
      const Unit w = unit_at(t, u, nk, bb);
      if constexpr (has_bat<Epi>::value) e.bat = bb;
      const int ntl = w.tile % t.grid_n, mt = (w.tile / t.grid_n) % t.grid_m, z = w.z;
      const int ntp = ntl < t.nt0 ? ntl : t.nt1_first + (ntl - t.nt0);
      const int64_t n0 = (int64_t)ntp * BN;
      const int my_nk = w.nk;
      const int buf = local & 1;
      const uint32_t use = (uint32_t)(local >> 1);
      if (!mbar_wait(&accf[buf], use & 1u, t.err)) break;
      tc_fence_after();
#pragma unroll 1
      for (int c = 0; c < BN; c += 16) {
        float v[16];
        if (my_nk > 0) {
          tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + c), v);
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = 0.f;
        }
        if constexpr (has_warp_tile<Epi>::value) {
#pragma unroll
          for (int k = 0; k < 16; ++k) stage[lane * 17 + k] = v[k];
          __syncwarp();
          e.warp_tile((int64_t)mt * BM + q * 32, n0 + c, z, stage, lane);
          __syncwarp();
        } else {
          e((int64_t)mt * BM + row, n0 + c, z, v);
        }
      }
      if constexpr (has_unit_end<Epi>::value) e.unit_end(q, w.tile);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[buf]);
    }
    e.done(q);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

// ------------------------------------------------------------------ host --

// Encodes a 2-D BF16 tensor map: `rows` rows of `cols` elements, row pitch
// `ld` elements (ld * 2 must be a multiple of 16), box = 64 x box_rows.
bool make_map_bf16(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows);
// The same over nb problems stored one after another (rows x ld elements
// each): a 3-D map whose third coordinate is the problem; rows past `rows`
// of a problem read as zero.
bool make_map_bf16_3d(CUtensorMap* map, const void* base, int64_t nb, int64_t rows, int64_t cols, int64_t ld,
                      int box_rows);

// Range bookkeeping shared by the launchers: K and N tiles that overlap the
// complement [0, lo) U [hi, p) of a set.
struct TileRanges {
  int r0_end, r1_begin, r1_end;
  int count() const { return r0_end + (r1_end - r1_begin); }
};
inline TileRanges complement_tiles(int64_t lo, int64_t hi, int64_t p, int tile) {
  TileRanges r;
  r.r0_end = (int)((lo + tile - 1) / tile);
  r.r1_begin = (int)(hi / tile);
  r.r1_end = (int)((p + tile - 1) / tile);
  if (r.r1_begin < r.r0_end) r.r1_begin = r.r0_end;
  if (r.r1_end < r.r1_begin) r.r1_end = r.r1_begin;
  return r;
}

// Resident CTAs of the persistent grid (SM count x CTAs per SM).
template <int S, int BN>
int resident_ctas() {
  static std::atomic<int> sms{0};
  if (sms.load() == 0) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    sms.store(n > 0 ? n : 148);
  }
  return sms.load() * Cfg<S, BN>::CTAS_PER_SM;
}

template <int S, int BN, class Epi>
cudaError_t launch(const Maps& maps, const Tiles& t0, int grid_n, int grid_m, const Epi& epi, cudaStream_t st,
                   int* grid_used = nullptr) {
  using C = Cfg<S, BN>;
  constexpr uint32_t smem_bytes = C::SMEM + (has_warp_tile<Epi>::value ? STAGE_TILE_BYTES : 0u);
  static_assert(smem_bytes <= 227 * 1024, "shared memory per CTA");
  static_assert(C::CTAS_PER_SM * (smem_bytes + 1024) <= 228 * 1024, "shared memory of the CTAs on an SM");
  static std::atomic<bool> attr_set{false};
  if (!attr_set.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<S, BN, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes);
    if (e != cudaSuccess) return e;
    attr_set.store(true, std::memory_order_release);
  }
  if (grid_used) *grid_used = 0;
  if (grid_n <= 0 || grid_m <= 0) return cudaSuccess;
  Tiles t = t0;
  t.grid_n = grid_n;
  t.grid_m = grid_m;
  const int64_t total = total_units(t);
  const int grid = (int)std::min<int64_t>(total, (int64_t)resident_ctas<S, BN>());
  if (grid_used) *grid_used = grid;
  note_launch();
  if (!t.pdl) {
    k_tc_gemm<S, BN, Epi><<<grid, THREADS, smem_bytes, st>>>(maps, t, epi);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = smem_bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_tc_gemm<S, BN, Epi>, maps, t, epi);
}

}  // namespace tc
}  // namespace ibmi
