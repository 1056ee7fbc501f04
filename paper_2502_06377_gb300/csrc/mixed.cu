// Mixed-precision IBMI sweep: the two sweep products (a3, a4) run on tcgen05
// tensor cores with BF16x3 operands (hi/lo slices, FP32 accumulation in TMEM);
// the iterate lives in HBM as an FP32 master plus its two BF16 slices, all
// updated in place by the GEMM epilogues.  The block invariants stay FP64.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <map>
#include <mutex>

#include "mixed.cuh"
#include "oz_rows.cuh"
#include "tail_plan.h"
#include "refine.cuh"
#include "tc_gemm.cuh"

namespace ibmi {

namespace tc {

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

bool make_map_bf16(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  auto enc = get_encode();
  if (!enc) return false;
  if (((uintptr_t)base & 15) != 0 || ((ld * 2) & 15) != 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_map_bf16_3d(CUtensorMap* map, const void* base, int64_t nb, int64_t rows, int64_t cols, int64_t ld,
                      int box_rows) {
  auto enc = get_encode();
  if (!enc) return false;
  if (((uintptr_t)base & 15) != 0 || ((ld * 2) & 15) != 0 || nb < 1) return false;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)nb};
  cuuint64_t strides[2] = {(cuuint64_t)(ld * 2), (cuuint64_t)(rows * ld * 2)};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace tc

constexpr int MX_BN = 128;   // N tile of the sweep products
constexpr int kRadiusIters = 40;            // power-iteration steps of the radius estimate
constexpr int kNsFirstGroups = 5;           // digit groups of a residual before the tail is calibrated
constexpr int kNsFixedFirst = 7;            // below kEarlyMinOrder: groups of the first tail residual ...
constexpr int kNsFixedNext = 8;             // ... and of the next ones while rho^2 > 1e3 tol
constexpr double kEarlyHandOver = 0.6;      // radius below which slow sweeps hand over early
constexpr int64_t kEarlyMinOrder = 2048;    // smallest order for that test
constexpr int64_t kTcInverseMinOrder = 512;    // block order from which Y^T Y runs on the tensor cores
constexpr double kRadiusHandOver = 0.5;     // hand over to Newton-Schulz below this radius

// One captured phase: the executable graph and its kernel-node count (added
// to the launch counter on every replay).
struct PhaseGraph {
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;
};

struct MixedState {
  int64_t ldp = 0;                       // padded row pitch of all mixed arrays (multiple of 64)
  float* Hf = nullptr;                   // FP32 master of H, p x ldp
  __nv_bfloat16* Hs[3] = {nullptr, nullptr, nullptr};   // BF16 slices of H: x ~ s0 + s1 + s2
  std::vector<__nv_bfloat16*> Ws[3];     // per set: BF16 slices of W (m x ldp)
  int level = 0;                         // sweep products: 0 = two slices (3 MMAs), 1 = three (6)
  float* Spart = nullptr;                // a4 split-K partial products, splits x mmax^2
  int splits_max = 0;
  int* err = nullptr;                    // device error word of the tcgen05 kernels
  CUtensorMap mapH[3];

  std::vector<CUtensorMap> mapW[3];
  void* pool = nullptr;
  double* Xprev = nullptr;               // p x p: the tail's iterate before its last update
  RefineState ref;                       // FP64-accurate residual + Newton-Schulz
  // CUDA graphs of the pipeline's phases (graph mode): captured on first use
  // for the A and H the plan was run with, replayed afterwards.
  bool graphs = false;
  const double* gA = nullptr;
  const double* gH = nullptr;
  PhaseGraph g_setup, g_sweep[2], g_cheap, g_reslice, g_export_resid, g_update[4], g_radius;
  std::map<int, PhaseGraph> g_tail;      // tail residuals by digit groups (see ns_graph_key)
};

static void drop_graphs(MixedState* M) {
  for (PhaseGraph* g : {&M->g_setup, &M->g_sweep[0], &M->g_sweep[1], &M->g_cheap, &M->g_reslice,
                        &M->g_export_resid, &M->g_update[0], &M->g_update[1], &M->g_update[2],
                        &M->g_update[3], &M->g_radius}) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    *g = PhaseGraph{};
  }
  for (auto& kv : M->g_tail)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  M->g_tail.clear();
}

// Newton-Schulz tail plan: tail_plan.h (host logic, tested on the CPU).
// graph keys of the tail's residuals: (export of H first, groups) and extensions (from, to)
static int ns_graph_key(bool export_h, int q) { return (export_h ? 100 : 0) + q; }
static int ns_extend_key(int qfrom, int qto) { return 200 + 10 * qfrom + qto; }
// ... and corrections (groups) and their extensions (from, to)
static int ns_correct_key(int q) { return 400 + q; }
static int ns_correct_extend_key(int qfrom, int qto) { return 500 + 10 * qfrom + qto; }

// Runs `body` (kernel launches only, no host synchronisation) directly, or in
// graph mode captures it once into *g and replays the graph.  While per-class
// profiling is on, launches are direct (its events are host-side records).
template <class F>
static ibmi_status graph_or_run(MixedState* M, PhaseGraph* g, cudaStream_t st, F&& body) {
  if (!M->graphs || prof_on()) return body();
  if (!g->exec) {   // the launches noted while capturing count the first run
    cudaGraph_t graph = nullptr;
    IBMI_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    const ibmi_status s = body();
    const cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (s != IBMI_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      if (s == IBMI_OK) set_last_error(std::string("graph capture: ") + cudaGetErrorString(e));
      return s != IBMI_OK ? s : IBMI_ERR_CUDA;
    }
    size_t n = 0;
    cudaGraphGetNodes(graph, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (n) cudaGraphGetNodes(graph, nodes.data(), &n);
    int kernels = 0;
    for (cudaGraphNode_t v : nodes) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(v, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
    }
    const cudaError_t ei = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      g->exec = nullptr;
      set_last_error(std::string("graph instantiate: ") + cudaGetErrorString(ei));
      return IBMI_ERR_CUDA;
    }
    g->kernels = kernels;
  } else {
    note_launch(g->kernels);
  }
  IBMI_CUDA_TRY(cudaGraphLaunch(g->exec, st));
  return IBMI_OK;
}

void mixed_enable_graphs(ibmi_plan_s* P, bool on) {
  MixedState* M = (MixedState*)P->mixed;
  if (!M) return;
  if (!on) drop_graphs(M);
  M->graphs = on;
}

static MixedState* MS(ibmi_plan_s* P) { return (MixedState*)P->mixed; }

// ------------------------------------------------------------- kernels ----


// FP64 H (ldh) -> FP32 master + BF16 hi/lo (ldp)
// Elementwise kernels run on 2-D grids: row = blockIdx.y, column =
// blockIdx.x * 256 + threadIdx.x (no 64-bit index division).
__global__ void k_import_h(const double* H, int64_t ldh, int64_t p, int64_t ldp, float* Hf, __nv_bfloat16* s0,
                           __nv_bfloat16* s1, __nv_bfloat16* s2) {
  const int64_t i = blockIdx.y, c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ldp) return;
  const int64_t idx = i * ldp + c;
  float x = c < p ? (float)H[i * ldh + c] : 0.f;
  Hf[idx] = x;
  split3(x, s0[idx], s1[idx], s2[idx]);
}

__global__ void k_export_h(const float* Hf, int64_t ldp, int64_t p, double* H, int64_t ldh) {
  const int64_t i = blockIdx.y, c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p) return;
  H[i * ldh + c] = (double)Hf[i * ldp + c];
}

// a4 finish: H[I, I] = A_I^{-1} - P with P = sum of the split-K partials (its
// lower triangle, mirrored).  One row per block row: the partials fit in L2
// (they were just written), so the mirrored half's column reads stay there;
// measured faster than 32 x 32 tiles through shared memory on 5120-row sets.
__global__ void k_mixed_sym(const float* Spart, int splits, int64_t m, const double* Ainv, int64_t lo, int64_t ldp,
                            float* Hf, __nv_bfloat16* s0, __nv_bfloat16* s1, __nv_bfloat16* s2) {
  const int64_t i = blockIdx.y, j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  // P is computed on and below the diagonal: element (max, min) serves both
  // (i, j) and (j, i), so H[I, I] comes out exactly symmetric
  const int64_t hi_ = i > j ? i : j, lo_ = i > j ? j : i;
  float a = 0.f;
  for (int z = 0; z < splits; ++z) a += Spart[(int64_t)z * m * m + hi_ * m + lo_];
  float x = (float)(Ainv[i * m + j] - (double)a);
  int64_t o = (lo + i) * ldp + lo + j;
  Hf[o] = x;
  __nv_bfloat16 t0, t1, t2;
  split3(x, t0, t1, t2);
  s0[o] = t0;
  s1[o] = t1;
  if (s2) s2[o] = t2;
}

static inline dim3 grid2(int64_t cols, int64_t rows) {
  return dim3((unsigned)((cols + 255) / 256), (unsigned)rows);
}

// All three slices of H from the FP32 master (entering the three-slice sweep).
__global__ void k_reslice_h(const float* Hf, int64_t n, __nv_bfloat16* s0, __nv_bfloat16* s1, __nv_bfloat16* s2) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  split3(Hf[idx], s0[idx], s1[idx], s2[idx]);
}

// a3 epilogue: X = -acc for rows i < m of the set and columns j in I^c,
// written to H[lo+i, j] and to H[j, lo+i].  The warp's 32 x 16 block comes
// through shared memory: the transposed copy goes out lane = row (32
// consecutive columns of H per store), the direct copy lane = (row 2k +
// lane/16, column lane%16) (two 16-wide row pieces per store).
struct EpiTcSweepX : tc::EpiBase {
  float* Hf; __nv_bfloat16* H0; __nv_bfloat16* H1; __nv_bfloat16* H2;
  int64_t ldp, lo, hi, p, m;
  __device__ __forceinline__ void put(int64_t idx, float x) const {
    __nv_bfloat16 a, b, d;
    split3(x, a, b, d);
    Hf[idx] = x;
    H0[idx] = a;
    H1[idx] = b;
    if (H2) H2[idx] = d;   // third slice only while the sweep uses three
  }
  __device__ __forceinline__ void warp_tile(int64_t row0, int64_t j0, int, const float* __restrict__ stage,
                                            int lane) const {
    {  // H[j, lo + i]: lane = row i
      const int64_t i = row0 + lane;
      if (i < m) {
#pragma unroll 4
        for (int c = 0; c < 16; ++c) {
          const int64_t j = j0 + c;
          if (j < p && (j < lo || j >= hi)) put(j * ldp + lo + i, -stage[lane * 17 + c]);
        }
      }
    }
    const int c = lane & 15;
    const int64_t j = j0 + c;
    if (j >= p || (j >= lo && j < hi)) return;
#pragma unroll 4
    for (int k = 0; k < 16; ++k) {   // H[lo + i, j]: lane = (row, column)
      const int r = 2 * k + (lane >> 4);
      const int64_t i = row0 + r;
      if (i < m) put((lo + i) * ldp + j, -stage[r * 17 + c]);
    }
  }
};

// a4 epilogue: split-K partial of X W^T, rows/cols < m, through shared memory
// so that each store covers 16 consecutive columns of two rows.
struct EpiTcPartial : tc::EpiBase {
  float* Spart; int64_t m;
  __device__ __forceinline__ void warp_tile(int64_t row0, int64_t j0, int z, const float* __restrict__ stage,
                                            int lane) const {
    const int c = lane & 15;
    if (j0 + c >= m) return;
    float* o = Spart + (int64_t)z * m * m + j0 + c;
#pragma unroll 4
    for (int k = 0; k < 16; ++k) {
      const int r = 2 * k + (lane >> 4);
      const int64_t i = row0 + r;
      if (i < m) o[i * m] = stage[r * 17 + c];
    }
  }
};

// a4 with one K split: the finish in the epilogue (no partials, no finishing
// kernel).  P = X W^T is computed on the tiles on and below the diagonal;
// each element (i, j), j <= i, gives x = A_I^{-1}[i, j] - P[i, j] (FP32),
// written to H[I, I] at (i, j) and, from the same x, at (j, i), so H[I, I]
// is exactly symmetric.  The first pass writes (i, j) along rows (16 columns
// of two rows per store) and keeps x in the warp's stage; the second writes
// (j, i) with one lane per row i, 32 consecutive columns of H's row j per
// store.
struct EpiTcSymFinish : tc::EpiBase {
  const double* Ainv; int64_t m, lo, ldp;
  float* Hf; __nv_bfloat16* s0; __nv_bfloat16* s1; __nv_bfloat16* s2;
  __device__ __forceinline__ void put(int64_t o, float x) const {
    Hf[o] = x;
    __nv_bfloat16 t0, t1, t2;
    split3(x, t0, t1, t2);
    s0[o] = t0;
    s1[o] = t1;
    if (s2) s2[o] = t2;
  }
  __device__ __forceinline__ void warp_tile(int64_t row0, int64_t j0, int, const float* __restrict__ stage_in,
                                            int lane) const {
    float* stage = const_cast<float*>(stage_in);   // this warp's own stage: x goes back in place
    const int c = lane & 15;
    const int64_t j = j0 + c;
    double a[16];   // all loads of A_I^{-1} in flight before the first store
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int64_t i = row0 + 2 * k + (lane >> 4);
      a[k] = i < m && j <= i ? Ainv[i * m + j] : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {   // (i, j): lane = (row, column), 16 columns of two rows per store
      const int r = 2 * k + (lane >> 4);
      const int64_t i = row0 + r;
      if (i < m && j <= i) {
        const float x = (float)(a[k] - (double)stage[r * 17 + c]);
        stage[r * 17 + c] = x;
        put((lo + i) * ldp + lo + j, x);
      }
    }
    __syncwarp();
    const int64_t i = row0 + lane;   // (j, i): lane = row i, consecutive in H's row j
#pragma unroll 4
    for (int cc = 0; cc < 16; ++cc) {
      const int64_t jj = j0 + cc;
      if (i < m && jj < i) put((lo + jj) * ldp + lo + i, stage[lane * 17 + cc]);
    }
  }
};

static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// --------------------------------------------------------------- host ----

ibmi_status mixed_create(ibmi_plan_s* P) {
  const int64_t p = P->d.p;
  const int K = (int)P->lo.size();
  MixedState* M = new MixedState();
  P->mixed = M;
  M->ldp = (p + 63) / 64 * 64;
  const int64_t ldp = M->ldp;
  // a4 split-K factor: fill one round of the SMs with the lower tiles
  const int64_t tm = (P->mmax + 127) / 128;
  const int64_t tiles2 = tm * (tm + 1) / 2;   // a4 computes the tiles on and below the diagonal
  int kt = (int)((p + tc::BK - 1) / tc::BK);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 148;
  M->splits_max = (int)std::max<int64_t>(1, std::min<int64_t>(std::max<int64_t>(1, sms / tiles2), kt / 4 > 0 ? kt / 4 : 1));
  size_t bytes = sizeof(float) * p * ldp + 3 * sizeof(__nv_bfloat16) * p * ldp + 512 +
                 sizeof(float) * (size_t)M->splits_max * P->mmax * P->mmax + 256 + sizeof(double) * p * p + 256;
  for (int k = 0; k < K; ++k) bytes += 3 * sizeof(__nv_bfloat16) * (P->hi[k] - P->lo[k]) * ldp + 768;
  if (cudaMalloc(&M->pool, bytes) != cudaSuccess) {
    cudaGetLastError();
    return IBMI_ERR_OOM;
  }
  uint8_t* q = (uint8_t*)M->pool;
  auto take = [&](size_t b) { uint8_t* r = q; q += (b + 255) / 256 * 256; return r; };
  M->Hf = (float*)take(sizeof(float) * p * ldp);
  for (int s = 0; s < 3; ++s) M->Hs[s] = (__nv_bfloat16*)take(sizeof(__nv_bfloat16) * p * ldp);
  M->Spart = (float*)take(sizeof(float) * (size_t)M->splits_max * P->mmax * P->mmax);
  M->err = (int*)take(256);
  M->Xprev = (double*)take(sizeof(double) * p * p);
  for (int k = 0; k < K; ++k) {
    const int64_t m = P->hi[k] - P->lo[k];
    for (int s = 0; s < 3; ++s) M->Ws[s].push_back((__nv_bfloat16*)take(sizeof(__nv_bfloat16) * m * ldp));
  }
  for (int s = 0; s < 3; ++s) {
    if (!tc::make_map_bf16(&M->mapH[s], M->Hs[s], p, p, ldp, 128)) return IBMI_ERR_CUDA;
    M->mapW[s].resize(K);
    for (int k = 0; k < K; ++k)
      if (!tc::make_map_bf16(&M->mapW[s][k], M->Ws[s][k], P->hi[k] - P->lo[k], p, ldp, 128)) return IBMI_ERR_CUDA;
  }
  IBMI_TRY(refine_create(&M->ref, p, M->err));
  return refine_plan_w(&M->ref, P->lo, P->hi);
}

void mixed_destroy(ibmi_plan_s* P) {
  MixedState* M = MS(P);
  if (!M) return;
  drop_graphs(M);
  refine_destroy(&M->ref);
  cudaFree(M->pool);
  delete M;
  P->mixed = nullptr;
}

ibmi_status mixed_prepare(ibmi_plan_s* P, const double* H, int64_t ldh, cudaStream_t st) {
  MixedState* M = MS(P);
  const int64_t p = P->d.p, ldp = M->ldp;
  ProfScope ps(IBMI_K_OTHER, st, 0.0);
  note_launch();
  k_import_h<<<grid2(ldp, p), 256, 0, st>>>(H, ldh, p, ldp, M->Hf, M->Hs[0], M->Hs[1], M->Hs[2]);
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

ibmi_status mixed_sweep_step(ibmi_plan_s* P, int k, cudaStream_t st) {
  MixedState* M = MS(P);
  const int64_t p = P->d.p, lo = P->lo[k], hi = P->hi[k], m = hi - lo, n = p - m;
  const tc::TileRanges kr = tc::complement_tiles(lo, hi, p, tc::BK);
  if (n == 0) return IBMI_ERR_INVALID_ARG;   // K = 1 never gets here (the FP64 path serves it)
  // a3: X = -W T; A operand = W slices (rows of the set), B = H slices (rows j).
  const int S = M->level == 0 ? 2 : 3;
  const double mult = S == 2 ? 3.0 : 6.0;   // slice products per product
  {
    // 128-wide N tiles.  (64-wide ones, which give small sets two tiles per
    // CTA so that one tile's epilogue runs under the other's MMAs, measured
    // slower on the 576-row sets of the p = 4096 workload, 31.2 against 23.0
    // ms per 10 inversions: they double the operand bytes per MMA.)
    const tc::TileRanges nr = tc::complement_tiles(lo, hi, p, MX_BN);
    tc::Maps maps;
    for (int s = 0; s < S; ++s) {
      maps.a[s] = M->mapW[s][k];
      maps.b[s] = M->mapH[s];
    }
    tc::Tiles t{m, 0, 0, nr.r0_end, nr.r1_begin, kr.r0_end, kr.r1_begin, kr.r1_end, 1, M->err};
    EpiTcSweepX epi{{}, M->Hf, M->Hs[0], M->Hs[1], S == 3 ? M->Hs[2] : nullptr, M->ldp, lo, hi, p, m};
    ProfScope ps(IBMI_K_SWEEP_X, st, mult * 2.0 * m * n * n, 2.0 * m * n * n);
    if (S == 2) IBMI_CUDA_TRY((tc::launch<2, MX_BN>(maps, t, nr.count(), (int)((m + 127) / 128), epi, st)));
    else IBMI_CUDA_TRY((tc::launch<3, MX_BN>(maps, t, nr.count(), (int)((m + 127) / 128), epi, st)));
  }
  // a4: P = X W^T (split over K); A operand = H slices rows [lo, hi), B = W slices.
  {
    const int nk = kr.count();
    // K splits to fill the SMs, but units of at least 12 K blocks (shorter
    // ones are all pipeline fill and partial store)
    const int splits = std::max(1, std::min(M->splits_max, nk / 12));
    tc::Maps maps;
    for (int s = 0; s < S; ++s) {
      maps.a[s] = M->mapH[s];
      maps.b[s] = M->mapW[s][k];
    }
    const int ntn = (int)((m + MX_BN - 1) / MX_BN);
    tc::Tiles t{m, lo, 0, ntn, ntn, kr.r0_end, kr.r1_begin, kr.r1_end, splits, M->err};
    t.lower = 1;   // P is symmetric up to rounding: tiles on and below the diagonal only
    ProfScope ps(IBMI_K_SWEEP_S, st, mult * 2.0 * n * (double)(ntn * (ntn + 1) / 2) * MX_BN * MX_BN,
                 2.0 * m * m * n);
    if (splits == 1) {   // the finish in the epilogue (no partials)
      EpiTcSymFinish epi{{}, P->ainv[k], m, lo, M->ldp, M->Hf, M->Hs[0], M->Hs[1], S == 3 ? M->Hs[2] : nullptr};
      if (S == 2) IBMI_CUDA_TRY((tc::launch<2, MX_BN>(maps, t, ntn, (int)((m + 127) / 128), epi, st)));
      else IBMI_CUDA_TRY((tc::launch<3, MX_BN>(maps, t, ntn, (int)((m + 127) / 128), epi, st)));
    } else {
      EpiTcPartial epi{{}, M->Spart, m};
      if (S == 2) IBMI_CUDA_TRY((tc::launch<2, MX_BN>(maps, t, ntn, (int)((m + 127) / 128), epi, st)));
      else IBMI_CUDA_TRY((tc::launch<3, MX_BN>(maps, t, ntn, (int)((m + 127) / 128), epi, st)));
      note_launch();
      k_mixed_sym<<<grid2(m, m), 256, 0, st>>>(M->Spart, splits, m, P->ainv[k], lo, M->ldp, M->Hf, M->Hs[0],
                                               M->Hs[1], S == 3 ? M->Hs[2] : nullptr);
      IBMI_CUDA_TRY(cudaGetLastError());
    }
  }
  return IBMI_OK;
}

static ibmi_status mixed_export_launch(ibmi_plan_s* P, double* H, int64_t ldh, cudaStream_t st) {
  MixedState* M = MS(P);
  const int64_t p = P->d.p;
  note_launch();
  k_export_h<<<grid2(p, p), 256, 0, st>>>(M->Hf, M->ldp, p, H, ldh);
  IBMI_CUDA_TRY(cudaGetLastError());
  return IBMI_OK;
}

ibmi_status mixed_run(ibmi_plan_s* P, const double* A, int64_t lda, double* H, int64_t ldh, cudaStream_t st,
                      ibmi_result* res, double* flops) {
  MixedState* M = MS(P);
  RefineState* R = &M->ref;
  const ibmi_plan_desc& d = P->d;
  const int64_t p = d.p;
  const int K = (int)P->lo.size();
  const double sqrtp = sqrt((double)p), fr = 2.0 * (double)p * p * p;
  double fs = 0.0, fplan = 0.0;
  for (int k = 0; k < K; ++k) {
    const double m = (double)(P->hi[k] - P->lo[k]), n = (double)p - m;
    fs += 2.0 * m * n * n + 2.0 * m * m * n;
    fplan += m * m * m / 3.0 + 2.0 * m * m * m + 2.0 * m * m * n;
  }
  if (M->graphs && (M->gA != A || M->gH != H)) {   // graphs bake in the buffers they were captured with
    drop_graphs(M);
    M->gA = A;
    M->gH = H;
  }
  // a2 (FP64 factorisations; W on tensor cores), the iterate and A's slices
  IBMI_TRY(graph_or_run(M, &M->g_setup, st, [&]() -> ibmi_status {
    IBMI_CUDA_TRY(cudaMemsetAsync(P->dstatus, 0, sizeof(DevStatus), st));
    IBMI_CUDA_TRY(cudaMemsetAsync(M->err, 0, sizeof(int), st));
    // Large blocks: A_I^{-1} = Y^T Y (Y = L^{-1}) as an exact sliced product
    // on the tensor cores instead of the FP64 product, which dominates there
    const bool tc_inverse = P->mmax >= kTcInverseMinOrder;
    IBMI_TRY(invariants_all(P, A, lda, false, st, tc_inverse, R));
    if (tc_inverse)   // all sets at once
      IBMI_TRY(refine_block_inverse_all(R, P->bat_R, P->mmax, K, P->pool, P->doff_ainv, P->dm, st));
    if (d.init == IBMI_INIT_IDENTITY) IBMI_TRY(set_identity(H, ldh, p, st));
    if (d.init == IBMI_INIT_SCHUR) IBMI_TRY(schur_guess_launch(P, A, lda, H, ldh, st, R));
    IBMI_TRY(refine_set_matrix(R, A, lda, st));
    if (R->w_rows > 0) {
      std::vector<const double*> ainv(P->ainv.begin(), P->ainv.end());
      IBMI_TRY(refine_form_w_all(R, ainv, P->lo, P->hi, M->Ws[0].data(), M->Ws[1].data(), M->Ws[2].data(), st));
    } else {
      for (int k = 0; k < K; ++k)
        IBMI_TRY(refine_form_w(R, P->ainv[k], P->hi[k] - P->lo[k], P->lo[k], P->hi[k], M->Ws[0][k], M->Ws[1][k],
                               M->Ws[2][k], st));
    }
    return mixed_prepare(P, H, ldh, st);
  }));
  *flops += fplan + (d.init == IBMI_INIT_SCHUR ? schur_guess_flops(P) : 0.0);
  IBMI_TRY(schur_guess_status(P, st, res));
  DevStatus hs;
  IBMI_CUDA_TRY(cudaMemcpyAsync(&hs, P->dstatus, sizeof(hs), cudaMemcpyDeviceToHost, st));
  IBMI_CUDA_TRY(cudaStreamSynchronize(st));
  if (hs.code == IBMI_ERR_NOT_SPD) {
    res->bad_block = hs.block;
    res->bad_pivot = hs.pivot;
    return IBMI_ERR_NOT_SPD;
  }
  M->level = 0;
  double pending = NAN;   // accurate residual of the current H when it was just taken
  double next_radius_test = INFINITY;   // slow convergence: rho below which the radius is measured again
  double handover_below = INFINITY;     // after a failed tail: rho below which the next hand-over may come
  double handover_rho = 0.0;            // rho of the stop test that handed over
  double last_cheap = INFINITY;         // rho of the last stop test of the sweeps
  // sweeps whose cost matches about two tail steps (time ratio of a step to a
  // sweep ~ 8.4 fr / fs, from the measured rates of the two kinds of product)
  const double slow_sweeps = 2.0 * 8.4 * fr / std::max(fs, 1.0);
  int r = 0, stalled = 0;
  double best = INFINITY;
  CheckCadence cad;
  cad.gmin = cad.next = d.check_every;
  const double target = d.ns_theta > 0.0 ? std::max(d.tol, d.ns_theta / sqrtp) : d.tol;
  auto accurate = [&](double* acc) -> ibmi_status {   // export H, FP64-accurate residual
    IBMI_TRY(graph_or_run(M, &M->g_export_resid, st, [&]() -> ibmi_status {
      IBMI_TRY(mixed_export_launch(P, H, ldh, st));
      return refine_residual_launch(R, H, ldh, st);
    }));
    *flops += fr;
    return refine_read(R, st, acc);
  };
  // From order kEarlyMinOrder the tail plans its residuals' digit groups on
  // the measured error model; below it launch latency, not the pair
  // products, sets a residual's cost, and a fixed schedule (no extension
  // round trips, few distinct graphs) does better.
  const bool planned = p >= kEarlyMinOrder;
  // A residual of the tail with digit groups <= q (exporting H first when
  // the sweeps just left it): its rho, the norm of group q's part and
  // ||A||_F ||X||_F / p.
  auto tail_residual = [&](bool export_h, int q, double* rho, double* g, double* amp) -> ibmi_status {
    IBMI_TRY(graph_or_run(M, &M->g_tail[ns_graph_key(export_h, q)], st, [&]() -> ibmi_status {
      if (export_h) IBMI_TRY(mixed_export_launch(P, H, ldh, st));
      return refine_residual_launch(R, H, ldh, st, q, planned);
    }));
    *flops += fr * tail::pairs(q, OZ_SX, OZ_SA) / tail::pairs(OZ_QMAX, OZ_SX, OZ_SA);
    return refine_read_groups(R, st, rho, g, amp);
  };
  // The same residual extended from groups <= qfrom to <= qto (only the new
  // groups' pair products run).
  auto tail_extend = [&](int qfrom, int qto, double* rho, double* g, double* amp) -> ibmi_status {
    IBMI_TRY(graph_or_run(M, &M->g_tail[ns_extend_key(qfrom, qto)], st,
                          [&]() { return refine_residual_extend_launch(R, H, ldh, st, qfrom, qto, planned); }));
    *flops += fr * (tail::pairs(qto, OZ_SX, OZ_SA) - tail::pairs(qfrom, OZ_SX, OZ_SA)) /
              tail::pairs(OZ_QMAX, OZ_SX, OZ_SA);
    return refine_read_groups(R, st, rho, g, amp);
  };
  // After an update from an exact residual (all groups, or a correction of
  // one): the residual of the new iterate from the previous one,
  // Q_X = Q_Xprev - (X - Xprev) A, with groups <= q of the digit products of
  // the small difference X - Xprev (its rho and the norm of group q's part).
  auto tail_correct = [&](int q, double* rho, double* g) -> ibmi_status {
    IBMI_TRY(graph_or_run(M, &M->g_tail[ns_correct_key(q)], st,
                          [&]() { return refine_residual_correct_launch(R, H, ldh, M->Xprev, st, q); }));
    *flops += fr * tail::pairs(q, OZ_SX, OZ_SA) / tail::pairs(OZ_QMAX, OZ_SX, OZ_SA);
    double unused;
    return refine_read_groups(R, st, rho, g, &unused);
  };
  auto tail_correct_extend = [&](int qfrom, int qto, double* rho, double* g) -> ibmi_status {
    IBMI_TRY(graph_or_run(M, &M->g_tail[ns_correct_extend_key(qfrom, qto)], st,
                          [&]() { return refine_residual_correct_extend_launch(R, st, qfrom, qto); }));
    *flops += fr * (tail::pairs(qto, OZ_SX, OZ_SA) - tail::pairs(qfrom, OZ_SX, OZ_SA)) /
              tail::pairs(OZ_QMAX, OZ_SX, OZ_SA);
    double unused;
    return refine_read_groups(R, st, rho, g, &unused);
  };
  // Before a radius test: the first tail residual's groups (q_first) give Q
  // ample for the radius and, if the tail starts, for its first step
  // (checked there); a value at or below tol is certified with all groups.
  const int q_first = planned ? kNsFirstGroups : kNsFixedFirst;
  double pending_g = NAN, pending_amp = NAN;
  int pending_q = 0;
  auto reduced = [&](double* acc) -> ibmi_status {
    pending_q = q_first;
    IBMI_TRY(tail_residual(true, pending_q, acc, &pending_g, &pending_amp));
    if (*acc <= d.tol) {
      IBMI_TRY(tail_extend(pending_q, OZ_QMAX, acc, &pending_g, &pending_amp));
      pending_q = OZ_QMAX;
    }
    return IBMI_OK;
  };
  // Sweeps, then the Newton-Schulz tail; a tail entered early that fails
  // returns here.
  for (;;) {
    bool early = false, resume = false;
    pending = NAN;
    while (true) {
      ++r;
      IBMI_TRY(graph_or_run(M, &M->g_sweep[M->level], st, [&]() -> ibmi_status {
        for (int k = 0; k < K; ++k) IBMI_TRY(mixed_sweep_step(P, k, st));
        return IBMI_OK;
      }));
      *flops += fs;
      res->sweeps = r;
      if (r < cad.next && r < d.max_sweeps) continue;
      double rho;
      IBMI_TRY(graph_or_run(M, &M->g_cheap, st, [&]() { return refine_cheap_residual_launch(R, M->mapH, st); }));
      IBMI_TRY(refine_read(R, st, &rho));
      *flops += fr;
      res->resid_f = rho;
      last_cheap = rho;
      if (!isfinite(rho)) return IBMI_ERR_NONFINITE;
      if (d.ns_theta > 0.0 && rho * sqrtp <= d.ns_theta && rho <= handover_below) {
        early = true;   // a failing tail returns to the sweeps
        handover_rho = rho;
        break;
      }
      // Slow convergence: eq. newton needs only the spectral radius of I - X A
      // below 1, which ||I - A H||_F bounds loosely.  Once that norm is within
      // 16 theta and the sweeps still predicted to reach theta cost more than
      // about two Newton-Schulz steps, measure the radius and hand over at
      // <= 0.6; otherwise test again after rho has halved.  A tail started this
      // way that fails returns to the sweeps (their state is untouched).  Below
      // order 2048 launch latency, not arithmetic, sets both costs and the
      // test (about 80 small launches) does not pay.
      if (d.ns_theta > 0.0 && p >= kEarlyMinOrder && rho * sqrtp <= 16.0 * d.ns_theta &&
          rho <= next_radius_test && cad.sweeps_to(rho, d.ns_theta / sqrtp) > slow_sweeps) {
        double acc, rad;
        IBMI_TRY(reduced(&acc));
        res->resid_f = acc;
        if (acc <= d.tol) return IBMI_OK;
        IBMI_TRY(graph_or_run(M, &M->g_radius, st, [&]() { return refine_q_radius_launch(R, kRadiusIters, st); }));
        *flops += 2.0 * kRadiusIters * (double)p * p;
        IBMI_TRY(refine_q_radius_read(R, st, &rad));
        next_radius_test = 0.5 * rho;
        if (rad <= kEarlyHandOver) {
          pending = acc;
          early = true;
          handover_rho = rho;
          break;
        }
      }
      // The sweep products have an accuracy floor (two BF16 slices: about
      // kappa(A) * 1e-5 in rho).  When the residual stops falling (three checks
      // without a 5% gain) the sweep first moves to three slices (24-bit
      // operands, six products); if it stalls there too, the Newton-Schulz
      // tail is tried when ||I - A H||_F is within 8 theta or the measured
      // spectral radius of I - X A is at most 1/2 (it stops if a step does not
      // help); otherwise the sweeps go on.
      stalled = rho > 0.95 * best ? stalled + 1 : 0;
      best = fmin(best, rho);
      if (d.ns_theta > 0.0 && stalled >= 3) {
        if (M->level == 0) {
          M->level = 1;
          stalled = 0;
          best = INFINITY;
          IBMI_TRY(graph_or_run(M, &M->g_reslice, st, [&]() -> ibmi_status {
            note_launch();
            k_reslice_h<<<nblk(p * M->ldp), 256, 0, st>>>(M->Hf, p * M->ldp, M->Hs[0], M->Hs[1], M->Hs[2]);
            IBMI_CUDA_TRY(cudaGetLastError());
            return IBMI_OK;
          }));
        } else if (rho * sqrtp <= 8.0 * d.ns_theta) {
          break;
        } else {
          // ||I - A H||_F bounds the spectral radius of I - X A that
          // eq. newton needs from above, often by far; measure the radius.
          double acc, rad;
          IBMI_TRY(reduced(&acc));
          res->resid_f = acc;
          if (acc <= d.tol) return IBMI_OK;
          IBMI_TRY(graph_or_run(M, &M->g_radius, st, [&]() { return refine_q_radius_launch(R, kRadiusIters, st); }));
          *flops += 2.0 * kRadiusIters * (double)p * p;
          IBMI_TRY(refine_q_radius_read(R, st, &rad));
          if (rad <= kRadiusHandOver) {
            pending = acc;
            break;
          }
          stalled = 0;
        }
      }
      if (rho <= d.tol || r >= d.max_sweeps) {
        // BF16x3 cannot certify tol: confirm with the FP64-accurate residual
        double acc;
        IBMI_TRY(accurate(&acc));
        res->resid_f = acc;
        if (acc <= d.tol) return IBMI_OK;
        if (r >= d.max_sweeps) return IBMI_NOT_CONVERGED;
      }
      cad.after(r, rho, target);
    }
    double prev = INFINITY, prev_floor = 0.0;
    double gcal = NAN, acal = NAN;   // calibration: norm of the last group of the last residual,
    int qcal = -1;                   // that group and ||A||_F ||X||_F / p
    bool exact = false;              // Q is exact for the iterate before the last update (planned tail)
    double amp_x = NAN;              // ||A||_F ||X||_F / p of the last direct residual
    for (int s = 0;; ++s) {
      double rho, g, amp = amp_x;
      int qc;
      bool corrected = false;
      if (s == 0 && !isnan(pending)) {
        rho = pending;
        g = pending_g;
        amp = pending_amp;
        qc = pending_q;
      } else if (s > 0 && planned && exact) {
        // from the exact residual of the previous iterate: groups until the
        // truncation is negligible against tol, for the value and for a step
        // it may feed (the correction's parts fall by about 2^-7 a group)
        qc = tail::kCorrectionGroups;
        IBMI_TRY(tail_correct(qc, &rho, &g));
        for (;;) {
          const int qn = isfinite(rho) ? tail::residual_groups(tail::kExactFraction * d.tol, g, qc, amp, qc, OZ_QMAX)
                                       : qc;
          if (qn == qc) break;
          IBMI_TRY(tail_correct_extend(qc, qn, &rho, &g));
          qc = qn;
        }
        corrected = true;
        exact = isfinite(rho) && tail::residual_floor(qc, g, qc, amp) <= tail::kExactFraction * d.tol;
      } else {
        // all groups where this residual is expected to certify tol; else
        // enough for the step it feeds, judged from the rho it should show
        const double rho_hat = s == 0 ? last_cheap : std::max(prev * prev, prev_floor);
        if (rho_hat <= d.tol) qc = OZ_QMAX;
        else if (!planned) qc = s == 0 ? kNsFixedFirst : (prev * prev > 1e3 * d.tol ? kNsFixedNext : OZ_QMAX);
        else
          qc = qcal < 0 ? kNsFirstGroups
                        : tail::residual_groups(tail::target(rho_hat, d.tol), gcal, qcal, acal, NS_S - 1, OZ_QMAX);
        IBMI_TRY(tail_residual(s == 0, qc, &rho, &g, &amp));
      }
      // a value at or below tol is certified with all groups; a step needs
      // the truncation error within its target (both extend the same residual)
      for (; !corrected;) {
        int qn = qc;
        if (rho <= d.tol || !isfinite(rho)) qn = isfinite(rho) ? OZ_QMAX : qc;
        else if (planned)
          qn = std::max(qc, tail::residual_groups(tail::target(rho, d.tol), g, qc, amp, NS_S - 1, OZ_QMAX));
        if (qn == qc) break;
        IBMI_TRY(tail_extend(qc, qn, &rho, &g, &amp));
        qc = qn;
      }
      if (!corrected) {
        exact = planned && qc == OZ_QMAX;
        amp_x = amp;
      }
      // the last update did not reduce the residual (or overflowed)
      const bool worse = s > 0 && !(rho < prev);
      if (!worse) {
        res->resid_f = rho;
        if (!isfinite(rho)) return IBMI_ERR_NONFINITE;
        if (rho <= d.tol) return IBMI_OK;
      }
      if (s >= d.ns_max || worse) {
        if (early && r < d.max_sweeps) {   // back to the sweeps (they re-export H)
          resume = true;
          break;
        }
        // H goes back to the better iterate before the failed update
        if (worse) IBMI_TRY(copy_square(H, ldh, M->Xprev, p, p, st));
        return IBMI_NOT_CONVERGED;
      }
      if (!corrected) {   // the calibration of the direct residuals
        gcal = g;
        acal = amp;
        qcal = qc;
      }
      // the update keeps 10 of its 15 pair products where their error fits
      // the same target as the residual's (planned tail only)
      const int qu = planned ? tail::update_groups(rho, amp, d.tol, NS_S - 1) : NS_S - 1;
      prev_floor = planned ? tail::residual_floor(qc, g, qc, amp) + tail::update_floor(qu, rho, amp) : 0.0;
      prev = rho;
      IBMI_TRY(graph_or_run(M, &M->g_update[(qu == NS_S - 1 ? 0 : 1) + (corrected ? 2 : 0)], st,
                            [&]() { return refine_ns_update(R, H, ldh, st, qu, M->Xprev, corrected, true); }));
      *flops += fr * tail::pairs(qu, NS_S, NS_S) / tail::pairs(NS_S - 1, NS_S, NS_S);
      res->ns_steps = s + 1;
    }
    if (!resume) return IBMI_NOT_CONVERGED;   // not reached: the tail returns
    // the next hand-over waits for rho to halve (the radius test's own
    // threshold was set when it ran)
    handover_below = 0.5 * handover_rho;
    cad.next = r + 1;
  }
}

// Epilogue of the wait self-test: never reached (no accumulator completes).
struct EpiNone : tc::EpiBase {
  __device__ __forceinline__ void operator()(int64_t, int64_t, int, const float (&)[16]) {}
};

}  // namespace ibmi

extern "C" ibmi_status ibmi_selftest_wait_timeout(void* stream) {
  using namespace ibmi;
  cudaStream_t st = (cudaStream_t)stream;
  // one 128 x 64 BF16 tile for the tensor maps (never loaded) and the error word
  constexpr size_t kTile = 128 * 64 * sizeof(__nv_bfloat16);
  void* buf = nullptr;
  IBMI_CUDA_TRY(cudaMalloc(&buf, kTile + 256));
  struct FreeOnExit {
    void* q;
    ~FreeOnExit() { cudaFree(q); }
  } keep{buf};
  int* err = (int*)((uint8_t*)buf + kTile);
  IBMI_CUDA_TRY(cudaMemsetAsync(buf, 0, kTile + 256, st));
  tc::Maps maps;
  for (int s = 0; s < 2; ++s)
    if (!tc::make_map_bf16(&maps.a[s], buf, 128, 64, 64, 128) || !tc::make_map_bf16(&maps.b[s], buf, 128, 64, 64, 128))
      return IBMI_ERR_CUDA;
  tc::Tiles t{128, 0, 0, 1, 0, 1, 1, 1, 1, err};
  t.starve = 1;
  IBMI_CUDA_TRY((tc::launch<2, 128>(maps, t, 1, 1, EpiNone{}, st)));
  int herr = 0;
  IBMI_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  IBMI_CUDA_TRY(cudaStreamSynchronize(st));
  if (herr == tc::ERR_TIMEOUT) {
    set_last_error("self-test: bounded wait expired as intended");
    return IBMI_ERR_TIMEOUT;
  }
  return herr == 0 ? IBMI_OK : IBMI_ERR_CUDA;
}
