// All slice-pair products of one error-free sliced product in a single
// persistent tcgen05 launch (internal).
//
// T_q += D_s(X) D_u(B)^T for every pair (s, u) of a list, in list order, each
// pair an exact FP32 accumulation in TMEM per K chunk (<= 4096 terms) that the
// epilogue adds in int32 into the digit-group plane T_q.  CTA c owns output
// tiles c, c + gridDim.x, ... for every pair, so all read-modify-writes of a
// tile come from one CTA in list order (no races), and the epilogue of one
// pair's last tile runs under the MMAs of the next pair's first tile: the
// pipeline fill, launch gap and exposed last epilogue of one launch per pair
// are gone.  Roles as in k_tc_gemm: warp 0 TMA producer, warp 1 MMA issuer,
// warps 2-5 epilogue through a shared-memory stage (row-coalesced int4).
#pragma once
#include <algorithm>

#include "oz_tiles.h"
#include "tc_gemm.cuh"

namespace ibmi {
namespace tc {

constexpr int OZP_MAX_A = 10, OZP_MAX_B = 8, OZP_MAX_PAIRS = 64;

struct OzPairMaps {
  CUtensorMap a[OZP_MAX_A];   // digit planes of the left operand (rows i), 128-row boxes
  CUtensorMap b[OZP_MAX_B];   // digit planes of the right operand (rows j), BN-row boxes
};

struct OzPairArgs {
  int n;                                   // pairs
  int8_t s[OZP_MAX_PAIRS], u[OZP_MAX_PAIRS], q[OZP_MAX_PAIRS], first[OZP_MAX_PAIRS];
  // Segments (oz_make_segments): runs of consecutive pairs of one group that
  // share one FP32 accumulation and one write of the group plane.
  int nseg;
  int8_t seg0[OZP_MAX_PAIRS], segn[OZP_MAX_PAIRS];
  int grid_n, tiles;                       // N tiles; tiles = grid_m * grid_n
  int kt_total, chunk;                     // K tiles; K tiles per exact accumulation
  int* T;                                  // group planes: T + q * plane, row pitch ldt
  int64_t plane, ldt, M, N;
  int* err;
  // Batch (nb > 0): 3-D maps with the problem as third coordinate; tiles of
  // problem bsel[i] (or i) follow those of the one before; group planes of
  // problem b at T + b * tstride.
  int nb;
  const int* bsel;
  int64_t tstride;
  // Optional per-problem digit-group ranges (indexed like bsel): the tiles of
  // problem i take only the pairs with qr[i].x <= q <= qr[i].y.
  const int2* qr;
  // Symmetric result (M == N): only the tiles that reach the diagonal or below
  // it are units, `tiles` of them (oz_lower_tiles), row by row.
  int lower;
  // Optional per-128-row-tile K-tile ranges [x, y) (one problem, no lower):
  // rows of different products stacked in one launch, each with its own K
  // range of at most `chunk` K tiles (kt_total = the longest, for the
  // segments' exactness bound).
  const int2* mkr;
};

static_assert(OZT_BM == BM, "lower-tile enumeration and the kernels' row tile");
using ibmi::oz_lower_row_tiles;
using ibmi::oz_lower_tiles;

// Output tile (mt, ntl) of tile index tl of a problem.
template <int BN>
__device__ __forceinline__ void oz_tile(const OzPairArgs& g, int tl, int& mt, int& ntl) {
  if (!g.lower) {
    mt = tl / g.grid_n;
    ntl = tl - mt * g.grid_n;
    return;
  }
  oz_lower_tile(tl, g.grid_n, BN, mt, ntl);
}

// Splits the pair list (in group order) into segments: a pair's product,
// summed over one K chunk of kc = min(K, 4096) terms, is an integer below
// kc 2^12 (digits of magnitude <= 64), so L = floor(4096 / kc) pairs of one
// group summed in FP32 stay below 2^24 and exact; they accumulate in TMEM
// together and the group plane is written once for them.
inline void oz_make_segments(OzPairArgs& g) {
  const int kc = std::min(g.kt_total, g.chunk) * BK;
  const int L = std::max(1, 4096 / std::max(1, kc));
  g.nseg = 0;
  for (int i = 0; i < g.n;) {
    int j = i + 1;
    while (j < g.n && j - i < L && g.q[j] == g.q[i]) ++j;
    g.seg0[g.nseg] = (int8_t)i;
    g.segn[g.nseg] = (int8_t)(j - i);
    ++g.nseg;
    i = j;
  }
}

// Whether unit tt (a tile of the problem at position bi) takes pair pi: the
// problem's digit-group range.  The same test in all three roles.
template <int BN>
__device__ __forceinline__ bool oz_pair_on(const OzPairArgs& g, int tt, int pi) {
  const int bi = tt / g.tiles;
  if (!g.qr) return true;
  const int2 r = g.qr[bi];
  return g.q[pi] >= r.x && g.q[pi] <= r.y;
}

template <int BN>
__global__ void __launch_bounds__(THREADS, Cfg<1, BN>::CTAS_PER_SM) k_oz_pairs(const __grid_constant__ OzPairMaps maps,
                                                         const __grid_constant__ OzPairArgs g) {
  using C = Cfg<1, BN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* tiles = smem;
  uint64_t* full = (uint64_t*)(smem + C::STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + C::STAGES;
  uint64_t* accf = empty + C::STAGES;
  uint64_t* acce = accf + 2;
  uint64_t* drain = acce + 2;   // MMA completion on an error exit
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunks = (g.kt_total + g.chunk - 1) / g.chunk;
  const int total = g.tiles * (g.nb > 0 ? g.nb : 1);   // tiles of all problems

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 4);
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
    if (lane == 0) {  // TMA producer
      int kc = 0;
      bool ok = true;
      for (int sg = 0; ok && sg < g.nseg; ++sg)
        for (int ci = 0; ok && ci < nchunks; ++ci)
          for (int tt = blockIdx.x; ok && tt < total; tt += gridDim.x) {
            const int bi = tt / g.tiles, tl = tt - bi * g.tiles;
            const int p0 = g.seg0[sg];
            if (!oz_pair_on<BN>(g, tt, p0)) continue;
            const int bb = g.bsel ? g.bsel[bi] : bi;
            int mt, ntl;
            oz_tile<BN>(g, tl, mt, ntl);
            int kb = ci * g.chunk, nk = min(g.chunk, g.kt_total - kb);
            if (g.mkr) {
              const int2 kr = g.mkr[mt];
              kb = kr.x;
              nk = kr.y - kr.x;
            }
            for (int j = 0; ok && j < g.segn[sg]; ++j) {
              const CUtensorMap* ma = &maps.a[g.s[p0 + j]];
              const CUtensorMap* mb = &maps.b[g.u[p0 + j]];
              for (int it = 0; it < nk; ++it, ++kc) {
                const int st = kc % C::STAGES;
                const uint32_t ph = (uint32_t)(kc / C::STAGES) & 1u;
                if (!mbar_wait(&empty[st], ph ^ 1u, g.err)) { ok = false; break; }
                const int kx = (kb + it) * BK;
                uint8_t* sa = tiles + st * C::STAGE_BYTES;
                mbar_expect_tx(&full[st], C::STAGE_BYTES);
                if (g.nb > 0) {
                  tma_load_3d(sa, ma, &full[st], kx, mt * BM, bb);
                  tma_load_3d(sa + C::A_BYTES, mb, &full[st], kx, ntl * BN, bb);
                } else {
                  tma_load_2d(sa, ma, &full[st], kx, mt * BM);
                  tma_load_2d(sa + C::A_BYTES, mb, &full[st], kx, ntl * BN);
                }
              }
            }
          }
      if (*(volatile int*)g.err != 0) {   // error exit: wait (bounded) for copies in flight
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
      int kc = 0, local = 0;
      bool ok = true;
      for (int sg = 0; ok && sg < g.nseg; ++sg)
        for (int ci = 0; ok && ci < nchunks; ++ci)
          for (int tt = blockIdx.x; ok && tt < total; tt += gridDim.x) {
            if (!oz_pair_on<BN>(g, tt, g.seg0[sg])) continue;
            int nk = min(g.chunk, g.kt_total - ci * g.chunk);
            if (g.mkr) {
              int mt, ntl;
              oz_tile<BN>(g, tt - (tt / g.tiles) * g.tiles, mt, ntl);
              nk = g.mkr[mt].y - g.mkr[mt].x;
            }
            const int buf = local & 1;
            const uint32_t use = (uint32_t)(local >> 1);
            if (!mbar_wait(&acce[buf], (use & 1u) ^ 1u, g.err)) { ok = false; break; }
            tc_fence_after();
            const uint32_t dacc = tmem + (uint32_t)(buf * BN);
            for (int j = 0; ok && j < g.segn[sg]; ++j)
              for (int it = 0; it < nk; ++it, ++kc) {
                const int st = kc % C::STAGES;
                const uint32_t ph = (uint32_t)(kc / C::STAGES) & 1u;
                if (!mbar_wait(&full[st], ph, g.err)) { ok = false; break; }
                tc_fence_after();
                const uint32_t sa = smem_u32(tiles + st * C::STAGE_BYTES);
                const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                  mma_bf16(dacc, sdesc_sw128(sa + kk * 32), sdesc_sw128(sb + kk * 32), idesc,
                           (j | it | kk) != 0 ? 1u : 0u);
                mma_commit(&empty[st]);
              }
            mma_commit(&accf[buf]);
            ++local;
          }
      if (!ok || *(volatile int*)g.err != 0) mma_drain_on_error(drain);
    }
  } else {  // epilogue warps 2..5
    const int qw = warp & 3;
    float* stage = (float*)(smem + C::STAGES * C::STAGE_BYTES + 256) + qw * 32 * 17;
    const int c4 = (lane & 3) * 4, r0 = lane >> 2;
    int local = 0;
    bool ok = true;
    for (int sg = 0; ok && sg < g.nseg; ++sg)
      for (int ci = 0; ok && ci < nchunks; ++ci)
        for (int tt = blockIdx.x; ok && tt < total; tt += gridDim.x) {
          const int pi = g.seg0[sg];   // the segment's first pair: its group and whether it stores
          const int bi = tt / g.tiles, tl = tt - bi * g.tiles;
          if (!oz_pair_on<BN>(g, tt, pi)) continue;
          const int bb = g.bsel ? g.bsel[bi] : bi;
          int mt, ntl;
          oz_tile<BN>(g, tl, mt, ntl);
          const int buf = local & 1;
          const uint32_t use = (uint32_t)(local >> 1);
          if (!mbar_wait(&accf[buf], use & 1u, g.err)) { ok = false; break; }
          tc_fence_after();
          int* Tq = g.T + (g.nb > 0 ? (int64_t)bb * g.tstride : 0) + (int64_t)g.q[pi] * g.plane;
          const bool first = g.first[pi] && ci == 0;
          const int64_t row0 = (int64_t)mt * BM + qw * 32;
#pragma unroll 1
          for (int c = 0; c < BN; c += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(qw * 32) << 16) + (uint32_t)(buf * BN + c), v);
#pragma unroll
            for (int k = 0; k < 16; ++k) stage[lane * 17 + k] = v[k];
            __syncwarp();
            // lane = (row 8k + lane/4, columns 4(lane%4)..+3): all staged values,
            // then all loads, then all stores
            const int64_t j0 = (int64_t)ntl * BN + c;
            int4 a[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const float* sv = stage + (8 * k + r0) * 17 + c4;
              a[k] = make_int4(__float2int_rn(sv[0]), __float2int_rn(sv[1]), __float2int_rn(sv[2]),
                               __float2int_rn(sv[3]));
            }
            __syncwarp();
            int* t0 = Tq + (row0 + r0) * g.ldt + j0 + c4;
            if (j0 + c4 + 4 <= g.N) {
              int4 o[4];
#pragma unroll
              for (int k = 0; k < 4; ++k)
                o[k] = (first || row0 + 8 * k + r0 >= g.M) ? make_int4(0, 0, 0, 0)
                                                            : *reinterpret_cast<const int4*>(t0 + 8 * k * g.ldt);
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                if (row0 + 8 * k + r0 >= g.M) continue;
                o[k].x += a[k].x;
                o[k].y += a[k].y;
                o[k].z += a[k].z;
                o[k].w += a[k].w;
                *reinterpret_cast<int4*>(t0 + 8 * k * g.ldt) = o[k];
              }
            } else {
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                if (row0 + 8 * k + r0 >= g.M) continue;
                int* t = t0 + 8 * k * g.ldt;
                const int vv[4] = {a[k].x, a[k].y, a[k].z, a[k].w};
                for (int uu = 0; uu < 4 && j0 + c4 + uu < g.N; ++uu) t[uu] = (first ? 0 : t[uu]) + vv[uu];
              }
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acce[buf]);
          ++local;
        }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

// Launches k_oz_pairs on min(tiles, SMs) persistent CTAs.
template <int BN>
cudaError_t launch_oz_pairs(const OzPairMaps& maps, const OzPairArgs& g, cudaStream_t st) {
  using C = Cfg<1, BN>;
  constexpr uint32_t smem_bytes = C::SMEM + STAGE_TILE_BYTES;
  static_assert(smem_bytes <= 227 * 1024, "shared memory per CTA");
  static_assert(C::CTAS_PER_SM * (smem_bytes + 1024) <= 228 * 1024, "shared memory of the CTAs on an SM");
  static std::atomic<bool> attr_set{false};
  if (!attr_set.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(k_oz_pairs<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) return e;
    attr_set.store(true, std::memory_order_release);
  }
  if (g.n <= 0 || g.tiles <= 0 || g.kt_total <= 0 || g.nseg <= 0) return cudaSuccess;
  const int grid = std::min(g.tiles * (g.nb > 0 ? g.nb : 1), resident_ctas<1, BN>());
  note_launch();
  k_oz_pairs<BN><<<grid, THREADS, smem_bytes, st>>>(maps, g);
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace ibmi
