// Mode B batched search: routing, bucketing, projection, Block-SoA scan,
// pool selection and exact rerank.
//
//   step                      paper                              kernel(s)
//   routing                   sec. 2.1 step 1, sec. 2.3 item 1   k_route_dist, k_route_select
//   (query, grain) bucketing  batched form of sec. 2.3 item 2    k_bucket_count/scan/scatter
//   projection                Eq. 1-4                            k_project
//   scan                      Eq. 6, sec. 2.1 step 3, sec. 2.4   k_scan_fp32
//   pool of C                 Table 1 "Pool C"                   k_select
//   exact rerank to k         sec. 2.1 step 4 (Mode B)           k_rerank
//
// Every distance is formed in direct difference form in FP32, the way the
// method states it: routing sum (q_t - mu_t)^2; projection of the centred
// query v' = q - mu_g; residual e = v' - U^T z and rho_q = ||e||^2; scan
// ||z_q - z_i||^2 + rho_q + rho_i; rerank sum (q_t - x_t)^2.
#include <cudaTypedefs.h>

#include <array>
#include <atomic>
#include <functional>
#include <cfloat>
#include <cstdint>
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "hntl_internal.cuh"
#include "kernels_common.cuh"
#include "route_kernels.cuh"
#include "scan_select.cuh"
#include "route_tc.cuh"
#include "project_tc.cuh"
#include "project_tc32.cuh"
#include "scan_tc.cuh"
#include "rerank.cuh"
#include "recon.cuh"

namespace hntl {

namespace {

// Test hook (hntl_debug_set_persistent_cap): when non-zero, the largest grid
// any persistent kernel of the search launches, so that small cases make every
// CTA loop over many work items the way full-size batches do.
std::atomic<uint32_t> g_persistent_cap{0};

// Grid of a persistent kernel that wants `want` CTAs (at least 1).
unsigned persistent_grid(size_t want) {
  const uint32_t cap = g_persistent_cap.load(std::memory_order_relaxed);
  if (cap && want > cap) want = cap;
  return (unsigned)std::max<size_t>(want, 1);
}

// ------------------------------------------------------------------ bounded-wait self test

// Waits, with the same bounded poll every tensor-core kernel uses, on an
// mbarrier whose phase nothing ever completes; after `polls` polls it gives
// up and records a timeout in the device error word, exactly as a stalled
// pipeline would, and returns.
__global__ void k_wait_selftest(uint32_t polls, int* __restrict__ err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, polls)) atomicOr(err, tc::kErrTimeout);
}

// ------------------------------------------------------------------ given probes

// Routing distance ||q - mu_g||^2 of caller-supplied probes (one warp per
// (query, probe); BF16-rounded values in the precision form). A grain id out
// of [0, G) is replaced by 0 and flagged in the device error word.
template <bool kBF16>
__global__ void k_probe_dist(const float* __restrict__ Q, const float* __restrict__ M, const uint16_t* __restrict__ Mh,
                             int nq, int nprobe, int G, int d, const int32_t* __restrict__ probe_in,
                             int32_t* __restrict__ probe, float* __restrict__ probe_d, int* __restrict__ err) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= nq * nprobe) return;
  int g = probe_in[w];
  if (g < 0 || g >= G) {
    if (lane == 0) atomicOr(err, 2);
    g = 0;
  }
  const float* q = Q + (size_t)(w / nprobe) * d;
  // the same arithmetic, in the same order, as the routing refine (warp_center_dist2)
  float acc = warp_center_dist2<kBF16>(
      [&](int t) { return kBF16 ? __bfloat162float(__float2bfloat16_rn(q[t])) : q[t]; }, M, Mh, g, d, lane);
  if (lane == 0) {
    probe[w] = g;
    probe_d[w] = acc;
  }
}

// ------------------------------------------------------------------ 16-bit form

// The 16-bit form's query side (Eq. 5, sec. 2.3), one warp per (query, grain)
// pair over the whole batch (a grain probed by many queries does not
// serialise), lanes over coordinates: each coordinate of z_q is put on the
// grain's grid, code rint(fl32(z / delta_g)) saturating at +-32767, and the
// codes, their squared sum and the grid values (for the scan's interval
// bound) are stored; rho_q goes on the residual grid, its code clipped at the
// unsigned 16-bit maximum 65535. A pair is left out (rho_q = +inf, residual
// code -1, so every downstream stage drops its rows) when more than a quarter
// of its coordinates saturate (the Quantization Envelope Filter), and, with
// the index's residual-saturation option (the library's own rule), when its
// residual code would exceed 65535.
__global__ void k_quant_pairs(uint32_t P, int nprobe, const int32_t* __restrict__ probe,
                              const uint32_t* __restrict__ pair_q, const uint32_t* __restrict__ pair_p, int r, int rp,
                              const float* __restrict__ delta, const float* __restrict__ dres, bool resid_prune,
                              float* __restrict__ zq, float* __restrict__ rhoq, int16_t* __restrict__ zq16,
                              long long* __restrict__ qn16, int32_t* __restrict__ rc16) {
  const uint32_t pr = (uint32_t)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (pr >= P) return;
  const int g = probe[(size_t)pair_q[pr] * nprobe + pair_p[pr]];
  const float dl = delta[g], dr = dres[g];
  float* z = zq + (size_t)pr * r;
  int sat = 0;
  long long qn = 0;
  for (int j0 = 0; j0 < rp; j0 += 32) {  // rp <= 64
    const int j = j0 + lane;
    float t = 0.f;
    if (j < r) t = rintf(z[j] / dl);
    const bool s = j < r && fabsf(t) > 32767.f;
    sat += __popc(__ballot_sync(0xffffffffu, s));
    const float c = fmaxf(-32767.f, fminf(32767.f, t));
    if (j < r) z[j] = c * dl;
    if (j < rp) zq16[(size_t)pr * rp + j] = (int16_t)c;
    const int ci = (int)c;
    qn += (long long)(ci * ci);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) qn += __shfl_xor_sync(0xffffffffu, qn, o);
  if (lane == 0) {
    float tr = rintf(rhoq[pr] / dr);
    bool out = 4 * sat > r;
    if (tr > 65535.f) {
      out = out || resid_prune;
      tr = 65535.f;
    }
    rhoq[pr] = out ? INFINITY : tr * dr;
    rc16[pr] = out ? -1 : (int32_t)tr;
    qn16[pr] = qn;
  }
}

// Diagnostic gather of the 16-bit query codes into query order: codes
// [nq][nprobe][r] and residual codes [nq][nprobe] (-1: pair left out).
__global__ void k_gather_pair_codes(uint32_t n, int r, int rp, const uint32_t* __restrict__ pair_of,
                                    const int16_t* __restrict__ zq16, const int32_t* __restrict__ rc16,
                                    int16_t* __restrict__ codes, int32_t* __restrict__ rcodes) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t pr = pair_of[i];
  for (int j = 0; j < r; ++j) codes[(size_t)i * r + j] = zq16[(size_t)pr * rp + j];
  rcodes[i] = rc16[pr];
}

// ------------------------------------------------------------------ bucketing

__global__ void k_bucket_count(const int32_t* __restrict__ probe, int n, uint32_t* __restrict__ gcnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&gcnt[probe[i]], 1u);
}

// Single CTA: exclusive scans over grains. Offsets of the grain-major pair
// lists, of the projection groups and of the 32-pair slots, and of the
// tensor-core scan's work items over the probed grains (scan_items ==
// nullptr skips them); k_bucket_fill then writes the slot table {grain,
// first pair, pairs} and the work items {grain, first block, blocks}.
__global__ void __launch_bounds__(1024) k_bucket_scan(const uint32_t* __restrict__ gcnt,
                                                      int G, uint32_t* __restrict__ pair_off,
                                                      uint32_t* __restrict__ grp_off,
                                                      uint32_t* __restrict__ slot_off, uint4* __restrict__ slots,
                                                      const uint32_t* __restrict__ blk_off,
                                                      uint32_t* __restrict__ scan_off,
                                                      uint4* __restrict__ scan_items) {
  // thread t owns grains [t per, (t + 1) per): one pass of local sums, one
  // block-wide scan of the four counts at once, then the offsets
  __shared__ uint4 wsum[32];
  __shared__ uint4 s_tot;
  const int per = (G + 1023) / 1024;  // G <= 8192: at most 8 grains per thread
  const int g0 = threadIdx.x * per;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto counts = [&](int g) {
    const uint32_t cnt = g < G ? gcnt[g] : 0u;
    const uint32_t nbk = (scan_items && g < G && cnt) ? blk_off[g + 1] - blk_off[g] : 0u;
    return make_uint4(cnt, (cnt + kPairsPerGroup - 1) / kPairsPerGroup, (cnt + kPSlot - 1) / kPSlot,
                      (nbk + kSTBlocks - 1) / kSTBlocks);
  };
  uint4 loc = make_uint4(0, 0, 0, 0);
  for (int i = 0; i < per; ++i) {
    const uint4 c = counts(g0 + i);
    loc.x += c.x;
    loc.y += c.y;
    loc.z += c.z;
    loc.w += c.w;
  }
  uint4 x = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t a = __shfl_up_sync(0xffffffffu, x.x, o), b = __shfl_up_sync(0xffffffffu, x.y, o);
    const uint32_t c = __shfl_up_sync(0xffffffffu, x.z, o), e = __shfl_up_sync(0xffffffffu, x.w, o);
    if (lane >= o) {
      x.x += a;
      x.y += b;
      x.z += c;
      x.w += e;
    }
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint4 v = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t a = __shfl_up_sync(0xffffffffu, v.x, o), b = __shfl_up_sync(0xffffffffu, v.y, o);
      const uint32_t c = __shfl_up_sync(0xffffffffu, v.z, o), e = __shfl_up_sync(0xffffffffu, v.w, o);
      if (lane >= o) {
        v.x += a;
        v.y += b;
        v.z += c;
        v.w += e;
      }
    }
    wsum[lane] = v;
    if (lane == 31) s_tot = v;
  }
  __syncthreads();
  const uint4 base = warp > 0 ? wsum[warp - 1] : make_uint4(0, 0, 0, 0);
  uint4 run = make_uint4(base.x + x.x - loc.x, base.y + x.y - loc.y, base.z + x.z - loc.z, base.w + x.w - loc.w);
  for (int i = 0; i < per; ++i) {
    const int g = g0 + i;
    if (g >= G) break;
    pair_off[g] = run.x;
    grp_off[g] = run.y;
    slot_off[g] = run.z;
    if (scan_items) scan_off[g] = run.w;
    const uint4 c = counts(g);
    run.x += c.x;
    run.y += c.y;
    run.z += c.z;
    run.w += c.w;
  }
  if (threadIdx.x == 0) {
    pair_off[G] = s_tot.x;
    grp_off[G] = s_tot.y;
    slot_off[G] = s_tot.z;
    if (scan_items) scan_off[G] = s_tot.w;
  }
}

// One thread per grain: the slot table and the scan work items from the
// offsets k_bucket_scan wrote (spread over the device rather than one CTA).
__global__ void k_bucket_fill(int G, const uint32_t* __restrict__ pair_off, const uint32_t* __restrict__ slot_off,
                              uint4* __restrict__ slots, const uint32_t* __restrict__ blk_off,
                              const uint32_t* __restrict__ scan_off, uint4* __restrict__ scan_items) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  if (slots) {
    const uint32_t p0 = pair_off[g], cnt = pair_off[g + 1] - p0, i0 = slot_off[g];
    for (uint32_t j = 0; j * kPSlot < cnt; ++j)
      slots[i0 + j] = make_uint4((uint32_t)g, p0 + j * kPSlot, min((uint32_t)kPSlot, cnt - j * kPSlot), 0u);
  }
  if (scan_items) {
    const uint32_t i0 = scan_off[g], n = scan_off[g + 1] - i0, bk0 = blk_off[g], nbk = blk_off[g + 1] - bk0;
    for (uint32_t j = 0; j < n; ++j)
      scan_items[i0 + j] =
          make_uint4((uint32_t)g, bk0 + j * kSTBlocks, min((uint32_t)kSTBlocks, nbk - j * kSTBlocks), 0u);
  }
}

__global__ void k_bucket_scatter(const int32_t* __restrict__ probe, int nq, int nprobe,
                                 const uint32_t* __restrict__ pair_off, uint32_t* __restrict__ gcur,
                                 uint32_t* __restrict__ pair_q, uint32_t* __restrict__ pair_p,
                                 uint32_t* __restrict__ pair_of, const float* __restrict__ probe_d,
                                 float* __restrict__ pair_vn) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq * nprobe) return;
  int g = probe[i];
  uint32_t pos = pair_off[g] + atomicAdd(&gcur[g], 1u);
  pair_q[pos] = (uint32_t)(i / nprobe);
  pair_p[pos] = (uint32_t)(i % nprobe);
  if (pair_vn) pair_vn[pos] = probe_d[i];
  pair_of[i] = pos;
}

// ------------------------------------------------------------------ host side

// Makes the index's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

struct Ws {
  float* qn;
  uint16_t* Qh;
  float* route_d;
  int32_t* probe;
  float* probe_d;
  uint32_t* gcnt;
  uint32_t* gcur;
  uint32_t* pair_off;
  uint32_t* grp_off;
  uint32_t* grp2_off;  // per-grain offsets of the 32-pair projection slots
  uint32_t* pair_q;
  uint32_t* pair_p;
  uint32_t* pair_of;
  float* pair_vn;  // ||q - mu_g||^2 of each pair (exact routing distance)
  uint4* slots;    // tensor-core projection slots of <= 32 pairs (precision form)
  uint32_t* scan_off;  // per-grain offsets of the tensor-core scan's work items (precision form)
  uint4* scan_items;   // {grain, first block, blocks} of each probed grain (precision form)
  uint4* dense_items;  // the items with many live pairs (tensor-core scan)
  uint32_t* need_list; // per grain, its pairs that can reach their pool (indices, at the grain's pair offset)
  uint32_t* need_cnt;  // per grain, how many
  SparseRec* sparse_items;  // the items with a few, with those pairs (direct-form scan)
  float* zq;
  float* rhoq;
  int16_t* zq16;     // 16-bit form: per-pair query codes [P][rp]
  long long* qn16;   // 16-bit form: per-pair sum of squared codes
  int32_t* rc16;     // 16-bit form: per-pair residual code (-1: left out)
  float* tau;
  uint32_t* cnt;
  unsigned long long* surv;
  uint32_t cap;
  uint32_t* cand_id;
  float* cand_d;
  size_t bytes;
};

Ws carve(const Index& I, uint32_t nq, uint32_t C, uint32_t nprobe, void* base) {
  Carver c(base);
  Ws w;
  const size_t P = (size_t)nq * nprobe;
  w.qn = c.take<float>(nq);
  w.Qh = I.precision == HNTL_PREC_BF16_FP8 ? c.take<uint16_t>((size_t)nq * I.d) : nullptr;
  w.route_d = c.take<float>((size_t)nq * I.G);
  w.probe = c.take<int32_t>(P);
  w.probe_d = c.take<float>(P);
  w.gcnt = c.take<uint32_t>(I.G);
  w.gcur = c.take<uint32_t>(I.G);
  w.pair_off = c.take<uint32_t>(I.G + 1);
  w.grp_off = c.take<uint32_t>(I.G + 1);
  w.grp2_off = c.take<uint32_t>(I.G + 1);
  w.pair_q = c.take<uint32_t>(P);
  w.pair_p = c.take<uint32_t>(P);
  w.pair_of = c.take<uint32_t>(P);
  const bool tcp = I.precision == HNTL_PREC_BF16_FP8;
  w.pair_vn = c.take<float>(P);  // the projection's ||v'||^2 (precision form) and Mode A's
  w.slots = (tcp || I.tc_proj32) ? c.take<uint4>(P / kPSlot + I.G) : nullptr;
  w.scan_off = tcp ? c.take<uint32_t>(I.G + 1) : nullptr;
  w.scan_items = tcp ? c.take<uint4>(I.G + I.n_blocks / kSTBlocks + 1) : nullptr;
  w.dense_items = tcp ? c.take<uint4>(I.G + I.n_blocks / kSTBlocks + 1) : nullptr;
  w.need_list = tcp ? c.take<uint32_t>(P) : nullptr;
  w.need_cnt = tcp ? c.take<uint32_t>(I.G) : nullptr;
  w.sparse_items = tcp ? c.take<SparseRec>(I.G + I.n_blocks / kSTBlocks + 1) : nullptr;
  w.zq = c.take<float>(P * I.r);
  w.rhoq = c.take<float>(P);
  const bool i16 = I.precision == HNTL_PREC_INT16;
  w.zq16 = i16 ? c.take<int16_t>(P * I.rp) : nullptr;
  w.qn16 = i16 ? c.take<long long>(P) : nullptr;
  w.rc16 = i16 ? c.take<int32_t>(P) : nullptr;
  w.tau = c.take<float>(nq);
  // survivor counts, then the scan's counters: [nq] next dense item, [nq + 1] dense items,
  // [nq + 2] light sparse items, [nq + 3] next sparse item, [nq + 4] heavy sparse items
  w.cnt = c.take<uint32_t>((size_t)nq + 5);
  w.cap = survivor_cap(C);
  w.surv = c.take<unsigned long long>((size_t)nq * w.cap);
  w.cand_id = c.take<uint32_t>((size_t)nq * C);
  w.cand_d = c.take<float>((size_t)nq * C);
  w.bytes = align_up(c.off, 256);
  return w;
}

int check_params(const Index& I, uint32_t nq, uint32_t k, uint32_t& C, uint32_t nprobe) {
  if (k < 1) return fail(HNTL_EINVAL, "k must be >= 1");
  if (C < k) C = k;
  if (C > (uint32_t)kMaxC) return fail(HNTL_EINVAL, "C (after raising it to k) must be <= 1024");
  if (nprobe < 1 || nprobe > I.G) return fail(HNTL_EINVAL, "nprobe must be in [1, G]");
  if ((uint64_t)nq * nprobe >= (1ull << 31)) return fail(HNTL_EINVAL, "nq * nprobe too large");
  return HNTL_OK;
}

// Centroid routing into w.probe / w.probe_d. With gcnt (zeroed), the
// tensor-core path also counts each grain's pairs there and sets *counted.
int launch_route(const Index& I, const float* Qd, uint32_t nq, uint32_t nprobe, const Ws& w, cudaStream_t st,
                 uint32_t* gcnt = nullptr, bool* counted = nullptr) {
  const bool bf16 = I.precision == HNTL_PREC_BF16_FP8;
  if (I.tc_route) {
    // tensor-core approximate distances, then the exact refine of a margin shortlist
    if (bf16) {  // d % 8 == 0 on this path (tensor-core routing)
      k_query_bf16<<<(nq * 32 + 255) / 256, 256, 0, st>>>(Qd, (int)nq, (int)I.d, w.Qh, w.qn);
    } else {
      k_row_norms<false><<<(nq * 32 + 255) / 256, 256, 0, st>>>(Qd, (int)nq, (int)I.d, w.qn);
    }
    CUtensorMap mapQ;
    if (!make_tma_map(&mapQ, bf16 ? (const void*)w.Qh : (const void*)Qd, bf16, nq, I.d, kRTM))
      return fail(HNTL_ECUDA, "cannot encode the TMA map of the queries");
    static thread_local int attr_tc = -1;
    if (attr_tc != I.device) {
      HNTL_CUDA_TRY(cudaFuncSetAttribute(k_route_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRouteTcSmem));
      HNTL_CUDA_TRY(cudaFuncSetAttribute(k_route_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRouteTcSmem));
      HNTL_CUDA_TRY(cudaFuncSetAttribute(k_route_refine<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kRefineSmemMax));
      HNTL_CUDA_TRY(cudaFuncSetAttribute(k_route_refine<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kRefineSmemMax));
      attr_tc = I.device;
    }
    // persistent: one CTA per SM at most
    const size_t tiles = (size_t)((I.G + kRTN - 1) / kRTN) * ((nq + kRTM - 1) / kRTM);
    const unsigned grid = persistent_grid(std::min<size_t>(tiles, (size_t)I.num_sms));
    const size_t rsmem = refine_smem_bytes((int)I.d, (int)I.G, (int)nprobe);
    float eps_dot = 0.f, eps_norm = 0.f;
    route_margin(bf16, (int)I.d, &eps_dot, &eps_norm);
    if (bf16) {
      k_route_tc<true><<<grid, kRThreads, kRouteTcSmem, st>>>(mapQ, I.mapM, (int)nq, (int)I.G, (int)I.d, w.qn, I.mnorm,
                                                        w.route_d, I.d_err);
      k_route_refine<true><<<nq, kRefineThreads, rsmem, st>>>(Qd, I.M, I.Mh, w.qn, I.mnorm, w.route_d, (int)I.G,
                                                              (int)I.d, (int)nprobe, eps_dot, eps_norm, w.probe,
                                                              w.probe_d, gcnt);
    } else {
      k_route_tc<false><<<grid, kRThreads, kRouteTcSmem, st>>>(mapQ, I.mapM, (int)nq, (int)I.G, (int)I.d, w.qn, I.mnorm,
                                                         w.route_d, I.d_err);
      k_route_refine<false><<<nq, kRefineThreads, rsmem, st>>>(Qd, I.M, I.Mh, w.qn, I.mnorm, w.route_d, (int)I.G,
                                                               (int)I.d, (int)nprobe, eps_dot, eps_norm, w.probe,
                                                               w.probe_d, gcnt);
    }
    HNTL_LAUNCH_CHECK("k_route_tc / k_route_refine");
    if (counted) *counted = gcnt != nullptr;
    return HNTL_OK;
  }
  if (bf16) return fail(HNTL_EINVAL, "the precision form needs tensor-core routing (d a multiple of 8)");
  dim3 grid((I.G + kRT - 1) / kRT, (nq + kRT - 1) / kRT);
  k_route_dist<<<grid, 256, 0, st>>>(Qd, I.M, (int)nq, (int)I.G, (int)I.d, w.route_d);
  size_t smem = (size_t)kSelWarps * I.G * sizeof(float);
  static thread_local int attr_sel = -1;  // device whose select attribute this thread has set
  if (attr_sel != I.device) {
    HNTL_CUDA_TRY(cudaFuncSetAttribute(k_route_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSelWarps * (int)kMaxG * (int)sizeof(float)));
    attr_sel = I.device;
  }
  k_route_select<<<(nq + kSelWarps - 1) / kSelWarps, kSelWarps * 32, smem, st>>>(w.route_d, (int)nq, (int)I.G,
                                                                                  (int)nprobe, w.probe, w.probe_d);
  HNTL_LAUNCH_CHECK("k_route_dist / k_route_select");
  return HNTL_OK;
}

template <int RN, bool kRho>
int launch_project_tc_n(const Index& I, uint32_t nq, uint32_t P, const Ws& w, cudaStream_t st) {
  static thread_local int attr_dev = -1;
  if (attr_dev != I.device) {
    HNTL_CUDA_TRY(cudaFuncSetAttribute(k_project_tc<RN, kRho>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       ProjTc<RN>::kSmem));
    attr_dev = I.device;
  }
  // persistent: one CTA per SM at most, never more CTAs than work items can exist
  const size_t max_items = ((size_t)P / kPSlot + I.G + kPSlots - 1) / kPSlots;
  const unsigned grid = persistent_grid(std::min<size_t>(max_items, (size_t)I.num_sms));
  k_project_tc<RN, kRho><<<grid, kPThreads, ProjTc<RN>::kSmem, st>>>(
      w.Qh, I.Mhn, I.mapU, I.gram, (int)I.d, (int)I.r, w.slots, w.grp2_off + I.G, w.pair_q, w.pair_vn, w.zq, w.rhoq,
      I.d_err);
  HNTL_LAUNCH_CHECK("k_project_tc");
  return HNTL_OK;
}

// The explicit residual rho_q = ||v' - U_b^T z||^2 of every pair (k_resid_tc),
// replacing the projection's Gram-identity value; bases of up to 32 rows.
template <int RN>
int launch_resid_tc_n(const Index& I, uint32_t P, const Ws& w, cudaStream_t st) {
  static thread_local int attr_dev = -1;
  if (attr_dev != I.device) {
    HNTL_CUDA_TRY(
        cudaFuncSetAttribute(k_resid_tc<RN>, cudaFuncAttributeMaxDynamicSharedMemorySize, ResidTc<RN>::kSmem));
    attr_dev = I.device;
  }
  const size_t max_items = ((size_t)P / kPSlot + I.G + kPSlots - 1) / kPSlots;
  const unsigned grid = persistent_grid(std::min<size_t>(max_items, (size_t)I.num_sms));
  k_resid_tc<RN><<<grid, kRThr, ResidTc<RN>::kSmem, st>>>(w.Qh, I.Mh, I.mapU, (int)I.d, (int)I.r, w.slots,
                                                          w.grp2_off + I.G, w.pair_q, w.zq, w.rhoq, I.d_err);
  HNTL_LAUNCH_CHECK("k_resid_tc");
  return HNTL_OK;
}

// The FP32-accurate projection of the FP32 and 16-bit forms: z (k_project_tc3),
// then the explicit residual (k_resid_tc3), over the precision form's items.
template <int RN>
int launch_project_tc32_n(const Index& I, const float* Qd, uint32_t P, const Ws& w, cudaStream_t st) {
  static thread_local int attr_dev = -1;
  if (attr_dev != I.device) {
    HNTL_CUDA_TRY(cudaFuncSetAttribute(k_project_tc3<RN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       ProjTc3<RN>::kSmem));
    HNTL_CUDA_TRY(
        cudaFuncSetAttribute(k_resid_tc3<RN>, cudaFuncAttributeMaxDynamicSharedMemorySize, ResidTc3<RN>::kSmem));
    attr_dev = I.device;
  }
  const size_t max_items = ((size_t)P / kPSlot + I.G + kPSlots - 1) / kPSlots;
  const unsigned grid = persistent_grid(std::min<size_t>(max_items, (size_t)I.num_sms));
  k_project_tc3<RN><<<grid, kP3Thr, ProjTc3<RN>::kSmem, st>>>(Qd, I.M, I.mapU3, (int)I.G, (int)I.d, (int)I.r,
                                                              w.slots, w.grp2_off + I.G, w.pair_q, w.zq, I.d_err);
  HNTL_LAUNCH_CHECK("k_project_tc3");
  k_resid_tc3<RN><<<grid, kR3Thr, ResidTc3<RN>::kSmem, st>>>(Qd, I.M, I.mapU3, (int)I.G, (int)I.d, (int)I.r,
                                                             w.slots, w.grp2_off + I.G, w.pair_q, w.zq, w.rhoq,
                                                             I.d_err);
  HNTL_LAUNCH_CHECK("k_resid_tc3");
  return HNTL_OK;
}

int launch_project_tc(const Index& I, uint32_t nq, uint32_t P, const Ws& w, cudaStream_t st) {
  if (!I.tc_proj) return fail(HNTL_EINVAL, "the precision form needs tensor-core projection (d a multiple of 8)");
  int rc;
  if (I.r <= 16) {
    if ((rc = launch_project_tc_n<16, false>(I, nq, P, w, st))) return rc;
    return launch_resid_tc_n<16>(I, P, w, st);
  }
  if (I.r <= 32) {
    if ((rc = launch_project_tc_n<32, false>(I, nq, P, w, st))) return rc;
    return launch_resid_tc_n<32>(I, P, w, st);
  }
  return launch_project_tc_n<64, true>(I, nq, P, w, st);  // r > 32: the Gram identity's rho_q
}

template <int RT, int kC>
void launch_scan_select(const Index& I, const Ws& w, int nq, int nprobe, int C, const int64_t* filter,
                        cudaStream_t st, const std::function<void(int)>& mark, const uint32_t* qC) {
  const Coords cz{I.Zb, I.Z8b, I.scale, I.Z16b};
  const I16Pairs q16{w.zq16, w.qn16};
  k_pilot<RT, kC><<<nq, 256, 0, st>>>(nprobe, C, w.probe, w.pair_of, I.blk_off, I.grain_rows, cz, I.rho,
                                        I.attr_b, (int)I.r, (int)I.rp, w.zq, w.rhoq, filter, w.tau, qC, q16);
  mark(4);
  if constexpr (kC == kCoordFP8) {
    static thread_local int attr_dev = -1;
    if (attr_dev != I.device) {
      cudaFuncSetAttribute(k_scan_tc<RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, ScanTc<RT>::kSmem);
      attr_dev = I.device;
    }
    const size_t max_items = (size_t)I.G + I.n_blocks / kSTBlocks + 1;
    uint32_t* lists = w.cnt + nq + 1;  // dense count, light sparse count, next sparse item, heavy sparse count
    k_grain_needed<<<I.G, 128, 0, st>>>(w.gcnt, w.pair_off, w.pair_q, w.rhoq, w.tau, I.grain_rho_min, w.need_list,
                                        w.need_cnt);
    k_scan_classify<<<(unsigned)((max_items * 32 + 255) / 256), 256, 0, st>>>(
        w.scan_items, w.scan_off + I.G, w.need_cnt, w.need_list, w.pair_off, w.pair_q, w.rhoq, w.tau, I.blk_rho_min,
        I.blk_z0, w.zq, (int)I.r, w.dense_items, w.sparse_items, (uint32_t)max_items, lists);
    k_scan_sparse<RT><<<persistent_grid(std::min<size_t>(max_items, (size_t)I.num_sms * 6)), kSPThreads, 0, st>>>(
        w.sparse_items, (uint32_t)max_items, lists, lists + 2, I.blk_off, I.grain_rows, I.Z8b, I.scale, I.rho, I.ids, I.attr_b, (int)I.r,
        (int)I.rp,
        w.pair_q, w.zq, w.rhoq, w.tau, I.blk_rho_min, I.blk_z0, filter, w.cap, w.cnt, w.surv);
    k_scan_tc<RT><<<persistent_grid(std::min<size_t>(max_items, (size_t)I.num_sms * 2)), kSTThreads, ScanTc<RT>::kSmem,
                    st>>>(
        w.dense_items, lists, w.cnt + nq, I.blk_off, I.grain_rows, I.Z8b, I.scale, I.crow, I.rho, I.ids, I.attr_b,
        (int)I.r, (int)I.rp, w.need_cnt, w.need_list, w.pair_off, w.pair_q, w.zq, w.rhoq, w.tau, I.blk_rho_min,
        filter, w.cap, w.cnt, w.surv, I.d_err);
  } else {
    k_scan_filter<RT, kC><<<(unsigned)I.n_blocks, kBlockRows, 0, st>>>(
        I.blk_grain, I.blk_off, I.grain_rows, cz, I.rho, I.ids, I.attr_b, (int)I.r, (int)I.rp, w.gcnt, w.pair_off,
        w.pair_q, w.zq, w.rhoq, w.tau, I.blk_rho_min, I.blk_z0, filter, w.cap, w.cnt, w.surv, q16);
  }
  mark(5);
  k_final_select<RT, kC, false><<<nq, kFinalThreads, 0, st>>>(
      nprobe, C, w.cap, w.cnt, w.surv, w.probe, w.pair_of, I.blk_off, I.grain_rows, cz, I.rho, I.ids, I.attr_b,
      (int)I.r, (int)I.rp, w.zq, w.rhoq, filter, w.cand_id, w.cand_d, qC, q16, (uint32_t)nq);
  const unsigned fb_grid =
      (unsigned)std::min<size_t>(((size_t)nq + kFinalThreads - 1) / kFinalThreads, (size_t)I.num_sms);
  k_final_select<RT, kC, true><<<fb_grid, kFinalThreads, 0, st>>>(
      nprobe, C, w.cap, w.cnt, w.surv, w.probe, w.pair_of, I.blk_off, I.grain_rows, cz, I.rho, I.ids, I.attr_b,
      (int)I.r, (int)I.rp, w.zq, w.rhoq, filter, w.cand_id, w.cand_d, qC, q16, (uint32_t)nq);
}

template <int RT>
void launch_scan_select_p(const Index& I, const Ws& w, int nq, int nprobe, int C, const int64_t* filter,
                          cudaStream_t st, const std::function<void(int)>& mark, const uint32_t* qC) {
  // FP8 rows are read in lanes of 16 codes, 16-bit rows in lanes of 8
  if (I.precision == HNTL_PREC_BF16_FP8)
    launch_scan_select<(RT < 16 ? 16 : RT), kCoordFP8>(I, w, nq, nprobe, C, filter, st, mark, qC);
  else if (I.precision == HNTL_PREC_INT16)
    launch_scan_select<(RT < 8 ? 8 : RT), kCoordI16>(I, w, nq, nprobe, C, filter, st, mark, qC);
  else
    launch_scan_select<RT, kCoordF32>(I, w, nq, nprobe, C, filter, st, mark, qC);
}

// Stage timing: CUDA events recorded on the search's stream between stages.
using StageEvents = std::array<cudaEvent_t, HNTL_NSTAGES + 1>;
struct Profiler {
  std::mutex mu;
  bool on = false;
  std::vector<StageEvents> pending, pool;
};
Profiler& profiler() {
  static Profiler p;
  return p;
}
bool profile_begin(StageEvents& ev) {
  Profiler& P = profiler();
  std::lock_guard<std::mutex> lk(P.mu);
  if (!P.on) return false;
  if (!P.pool.empty()) {
    ev = P.pool.back();
    P.pool.pop_back();
    return true;
  }
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) return false;
  return true;
}
void profile_end(const StageEvents& ev) {
  Profiler& P = profiler();
  std::lock_guard<std::mutex> lk(P.mu);
  P.pending.push_back(ev);
}

}  // namespace

int search(const Index& I, const float* Qd, uint32_t nq, uint32_t k, uint32_t C, uint32_t nprobe,
           const int64_t* filter, void* ws, size_t ws_bytes, int64_t* out_ids, float* out_d, uint32_t* cand_ids,
           float* cand_d, int32_t* probe_out, cudaStream_t st, const int32_t* probe_in = nullptr,
           const uint32_t* qk = nullptr, const uint32_t* qC = nullptr, bool mode_a = false) {
  int rc = check_params(I, nq, k, C, nprobe);
  if (rc) return rc;
  if (filter && !I.has_attr) return fail(HNTL_EINVAL, "filter given but the index has no attribute column");
  if (mode_a && I.precision == HNTL_PREC_INT16)
    return fail(HNTL_EINVAL, "Mode A is not available for the 16-bit form");
  if (!mode_a && !I.X && !I.Xh)
    return fail(HNTL_EINVAL, "the index was loaded without its raw rows: only Mode A can search it");
  if (nq == 0) return HNTL_OK;
  if (!Qd || !ws || !out_ids || !out_d) return fail(HNTL_EINVAL, "null buffer");
  if ((cand_ids == nullptr) != (cand_d == nullptr)) return fail(HNTL_EINVAL, "pass both pool buffers or neither");
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(HNTL_EINVAL, "workspace must be 256-byte aligned");
  Ws w = carve(I, nq, C, nprobe, ws);
  if (ws_bytes < w.bytes) return fail(HNTL_EINVAL, "workspace too small");
  if (cand_ids) {
    w.cand_id = cand_ids;
    w.cand_d = cand_d;
  }
  DeviceGuard dg(I.device);
  if (!dg.ok) return fail(HNTL_ECUDA, "cannot make the index's device current");
  StageEvents ev;
  const bool prof = profile_begin(ev);
  auto mark = [&](int i) {
    if (prof) cudaEventRecord(ev[i], st);
  };
  mark(0);
  HNTL_CUDA_TRY(cudaMemsetAsync(w.gcnt, 0, sizeof(uint32_t) * I.G, st));
  HNTL_CUDA_TRY(cudaMemsetAsync(w.gcur, 0, sizeof(uint32_t) * I.G, st));
  bool counted = false;  // the routing refine counted each grain's pairs
  if (probe_in) {
    const bool bf16 = I.precision == HNTL_PREC_BF16_FP8;
    if (bf16) {
      const size_t n = (size_t)nq * I.d;
      k_to_bf16_rows<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Qd, n, w.Qh);
    }
    const unsigned blocks = (unsigned)(((size_t)nq * nprobe * 32 + 255) / 256);
    if (bf16)
      k_probe_dist<true><<<blocks, 256, 0, st>>>(Qd, I.M, I.Mh, (int)nq, (int)nprobe, (int)I.G, (int)I.d, probe_in,
                                                w.probe, w.probe_d, I.d_err);
    else
      k_probe_dist<false><<<blocks, 256, 0, st>>>(Qd, I.M, I.Mh, (int)nq, (int)nprobe, (int)I.G, (int)I.d, probe_in,
                                                 w.probe, w.probe_d, I.d_err);
    HNTL_CUDA_TRY(cudaGetLastError());
  } else if ((rc = launch_route(I, Qd, nq, nprobe, w, st, w.gcnt, &counted))) {
    return rc;
  }
  mark(1);
  const int P = (int)(nq * nprobe);
  if (!counted) k_bucket_count<<<(P + 255) / 256, 256, 0, st>>>(w.probe, P, w.gcnt);
  k_bucket_scan<<<1, 1024, 0, st>>>(w.gcnt, (int)I.G, w.pair_off, w.grp_off, w.grp2_off, w.slots, I.blk_off,
                                    w.scan_off, w.scan_items);
  if (w.slots || w.scan_items)
    k_bucket_fill<<<(I.G + 255) / 256, 256, 0, st>>>((int)I.G, w.pair_off, w.grp2_off, w.slots, I.blk_off, w.scan_off,
                                                     w.scan_items);
  k_bucket_scatter<<<(P + 255) / 256, 256, 0, st>>>(w.probe, (int)nq, (int)nprobe, w.pair_off, w.gcur, w.pair_q,
                                                    w.pair_p, w.pair_of, w.probe_d, w.pair_vn);
  mark(2);
  if (I.precision == HNTL_PREC_BF16_FP8) {
    if ((rc = launch_project_tc(I, nq, (uint32_t)P, w, st))) return rc;
  } else {
    if (I.tc_proj32) {
      if ((rc = I.r <= 16 ? launch_project_tc32_n<16>(I, Qd, (uint32_t)P, w, st)
                          : launch_project_tc32_n<32>(I, Qd, (uint32_t)P, w, st)))
        return rc;
    } else {  // bases of more than 32 rows (or d not a multiple of 8): the direct form on the SIMT cores
      size_t smem = (size_t)kPairsPerGroup * I.d * sizeof(float);
      if (smem > 40 * 1024)  // the kernel's static shared memory counts against the default 48 KB too
        HNTL_CUDA_TRY(cudaFuncSetAttribute(k_project<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      unsigned grid = persistent_grid(std::min<size_t>((size_t)P / kPairsPerGroup + I.G, (size_t)I.num_sms * 16));
      k_project<false><<<grid, 256, smem, st>>>(Qd, I.M, I.U, (int)I.d, (int)I.r, (int)I.G, w.grp_off, w.pair_off,
                                                w.pair_q, w.zq, w.rhoq);
    }
    if (I.precision == HNTL_PREC_INT16)
      k_quant_pairs<<<(unsigned)(((size_t)P * 32 + 255) / 256), 256, 0, st>>>(
          (uint32_t)P, (int)nprobe, w.probe, w.pair_q, w.pair_p, (int)I.r, (int)I.rp, I.scale, I.dres,
          I.i16_resid_prune, w.zq, w.rhoq, w.zq16, w.qn16, w.rc16);
  }
  mark(3);
  HNTL_CUDA_TRY(cudaMemsetAsync(w.cnt, 0, sizeof(uint32_t) * ((size_t)nq + 5), st));
  {
    const std::function<void(int)> mk = mark;
    if (I.r <= 8) launch_scan_select_p<8>(I, w, (int)nq, (int)nprobe, (int)C, filter, st, mk, qC);
    else if (I.r <= 16) launch_scan_select_p<16>(I, w, (int)nq, (int)nprobe, (int)C, filter, st, mk, qC);
    else if (I.r <= 32) launch_scan_select_p<32>(I, w, (int)nq, (int)nprobe, (int)C, filter, st, mk, qC);
    else launch_scan_select_p<64>(I, w, (int)nq, (int)nprobe, (int)C, filter, st, mk, qC);
  }
  mark(6);
  if (mode_a) {
    const Coords cz{I.Zb, I.Z8b, I.scale, I.Z16b};
    auto recon = [&](auto kern) {
      kern<<<nq, 256, 0, st>>>((int)nprobe, (int)C, (int)k, w.cand_id, I.pos_of_id, I.blk_grain, cz, (int)I.r,
                               (int)I.rp, I.hrow, w.probe, w.pair_of, w.zq, w.pair_vn, out_ids, out_d, qk, qC);
    };
    if (I.precision == HNTL_PREC_BF16_FP8) {
      if (I.r <= 16) recon(k_rerank_recon<16, kCoordFP8>);
      else if (I.r <= 32) recon(k_rerank_recon<32, kCoordFP8>);
      else recon(k_rerank_recon<64, kCoordFP8>);
    } else {
      if (I.r <= 8) recon(k_rerank_recon<8, kCoordF32>);
      else if (I.r <= 16) recon(k_rerank_recon<16, kCoordF32>);
      else if (I.r <= 32) recon(k_rerank_recon<32, kCoordF32>);
      else recon(k_rerank_recon<64, kCoordF32>);
    }
  } else {
    size_t smem = (size_t)I.d * sizeof(float);
    if (smem > 40 * 1024) {
      HNTL_CUDA_TRY(cudaFuncSetAttribute(k_rerank<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      HNTL_CUDA_TRY(cudaFuncSetAttribute(k_rerank<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      HNTL_CUDA_TRY(
          cudaFuncSetAttribute(k_rerank<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    if (I.precision == HNTL_PREC_BF16_FP8 && I.Xl)  // refined: a second stage on both BF16 parts
      k_rerank<true, true><<<nq, 256, smem, st>>>(Qd, I.Xh, (int)I.d, (int)C, (int)k, w.cand_id, out_ids, out_d, qk,
                                                  qC, I.Xl);
    else if (I.precision == HNTL_PREC_BF16_FP8)
      k_rerank<true><<<nq, 256, smem, st>>>(Qd, I.Xh, (int)I.d, (int)C, (int)k, w.cand_id, out_ids, out_d, qk, qC);
    else
      k_rerank<false><<<nq, 256, smem, st>>>(Qd, I.X, (int)I.d, (int)C, (int)k, w.cand_id, out_ids, out_d, qk, qC);
  }
  mark(7);
  if (prof) profile_end(ev);
  if (probe_out)
    HNTL_CUDA_TRY(cudaMemcpyAsync(probe_out, w.probe, sizeof(int32_t) * nq * nprobe, cudaMemcpyDeviceToDevice, st));
  HNTL_CUDA_TRY(cudaGetLastError());
  return HNTL_OK;
}

size_t workspace_bytes(const Index& I, uint32_t nq, uint32_t k, uint32_t C, uint32_t nprobe) {
  if (check_params(I, nq, k, C, nprobe)) return 0;
  return carve(I, nq, C, nprobe, nullptr).bytes;
}

int route_only(const Index& I, const float* Qd, uint32_t nq, uint32_t nprobe, void* ws, size_t ws_bytes,
               int32_t* probe, float* probe_d, cudaStream_t st) {
  uint32_t C = 1;
  int rc = check_params(I, nq, 1, C, nprobe);
  if (rc) return rc;
  if (nq == 0) return HNTL_OK;
  if (!Qd || !ws || !probe || !probe_d) return fail(HNTL_EINVAL, "null buffer");
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(HNTL_EINVAL, "workspace must be 256-byte aligned");
  Ws w = carve(I, nq, C, nprobe, ws);
  if (ws_bytes < w.bytes) return fail(HNTL_EINVAL, "workspace too small");
  w.probe = probe;
  w.probe_d = probe_d;
  DeviceGuard dg(I.device);
  if (!dg.ok) return fail(HNTL_ECUDA, "cannot make the index's device current");
  return launch_route(I, Qd, nq, nprobe, w, st);
}

bool make_tma_map(CUtensorMap* map, const void* base, bool bf16, uint64_t rows, uint64_t d, uint32_t box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!encode || rows == 0) return false;
  const uint64_t elem = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(d * elem)};
  cuuint32_t box[2] = {(cuuint32_t)(128 / elem), box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                      const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int finalize_index(Index& I) {
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
    I.allocations.push_back(p);
    I.device_bytes += std::max<size_t>(bytes, 16);
    return p;
  };
  const bool bf16 = I.precision == HNTL_PREC_BF16_FP8;
  I.d_err = static_cast<int*>(alloc(sizeof(int)));
  I.mnorm = static_cast<float*>(alloc(sizeof(float) * I.G));
  I.gram = static_cast<float*>(alloc(sizeof(float) * I.G * I.r * I.r));
  I.pos_of_id = static_cast<uint32_t*>(alloc(sizeof(uint32_t) * std::max<uint64_t>(I.n, 1)));
  I.hrow = static_cast<float*>(alloc(sizeof(float) * I.n_blocks * kBlockRows));
  I.blk_z0 = static_cast<float2*>(alloc(sizeof(float2) * std::max<uint64_t>(I.n_blocks, 1)));
  if (bf16) {
    I.Mh = static_cast<uint16_t*>(alloc(sizeof(uint16_t) * I.G * I.d));
    I.Mhn = static_cast<uint16_t*>(alloc(sizeof(uint16_t) * I.G * I.d));
    I.Uh = static_cast<uint16_t*>(alloc(sizeof(uint16_t) * I.G * I.r * I.d));
    I.crow = static_cast<float*>(alloc(sizeof(float) * I.n_blocks * kBlockRows));
    I.grain_rho_min = static_cast<float*>(alloc(sizeof(float) * I.G));
  }
  // the FP32-accurate tensor-core projection: bases of up to 32 rows, 16-byte
  // row strides, the item's centre rows within its shared-memory stage
  const bool tc32_shape = !bf16 && I.r <= 32 && I.d % 8 == 0 && I.d <= (uint32_t)kP3MuD && I.G > 0;
  if (tc32_shape) I.U3 = static_cast<uint16_t*>(alloc(sizeof(uint16_t) * 3 * I.G * I.r * I.d));
  if (!I.d_err || !I.mnorm || !I.gram || !I.pos_of_id || !I.hrow || !I.blk_z0 ||
      (bf16 && (!I.Mh || !I.Mhn || !I.Uh || !I.crow || !I.grain_rho_min)) || (tc32_shape && !I.U3))
    return fail(HNTL_ENOMEM, "index: derived arrays");
  if (tc32_shape) {
    const size_t nu = (size_t)I.G * I.r * I.d;
    k_split3_bf16<<<(unsigned)std::min<size_t>((nu + 255) / 256, 65535), 256>>>(I.U, nu, I.U3);
  }
  HNTL_CUDA_TRY(cudaMemset(I.d_err, 0, sizeof(int)));
  if (bf16) k_row_norms<true><<<(I.G * 32 + 255) / 256, 256>>>(I.M, (int)I.G, (int)I.d, I.mnorm);
  else k_row_norms<false><<<(I.G * 32 + 255) / 256, 256>>>(I.M, (int)I.G, (int)I.d, I.mnorm);
  if (bf16) {
    const size_t n = (size_t)I.G * I.d, nu = (size_t)I.G * I.r * I.d;
    k_to_bf16_rows<<<(unsigned)((n + 255) / 256), 256>>>(I.M, n, I.Mh);
    k_to_bf16_rows_neg<<<(unsigned)((n + 255) / 256), 256>>>(I.M, n, I.Mhn);
    k_to_bf16_rows<<<(unsigned)((nu + 255) / 256), 256>>>(I.U, nu, I.Uh);
    k_gram<<<I.G, 256>>>(I.Uh, (int)I.d, (int)I.r, I.gram);  // of the BF16 bases the precision form uses
    k_grain_rho_min<<<(I.G * 32 + 255) / 256, 256>>>(I.blk_rho_min, I.blk_off, (int)I.G, I.grain_rho_min);
    const Coords cz{I.Zb, I.Z8b, I.scale, I.Z16b};
    if (I.n_blocks) {
      if (I.r <= 16) k_row_c<16><<<(unsigned)I.n_blocks, kBlockRows>>>(cz, I.rho, I.blk_grain, (int)I.rp, I.crow);
      else if (I.r <= 32) k_row_c<32><<<(unsigned)I.n_blocks, kBlockRows>>>(cz, I.rho, I.blk_grain, (int)I.rp, I.crow);
      else k_row_c<64><<<(unsigned)I.n_blocks, kBlockRows>>>(cz, I.rho, I.blk_grain, (int)I.rp, I.crow);
    }
  }
  // every block's interval of decoded first coordinates (the scan's interval bound)
  if (I.n_blocks) {
    const Coords cz{I.Zb, I.Z8b, I.scale, I.Z16b};
    const unsigned nb = (unsigned)I.n_blocks;
    const int rp = (int)I.rp;
    auto z0 = [&](auto kern) { kern<<<nb, kBlockRows>>>(cz, I.blk_grain, I.blk_off, I.grain_rows, rp, I.blk_z0); };
    if (bf16) {
      if (I.r <= 16) z0(k_block_z0<16, kCoordFP8>);
      else if (I.r <= 32) z0(k_block_z0<32, kCoordFP8>);
      else z0(k_block_z0<64, kCoordFP8>);
    } else if (I.precision == HNTL_PREC_INT16) {
      if (I.r <= 8) z0(k_block_z0<8, kCoordI16>);
      else if (I.r <= 16) z0(k_block_z0<16, kCoordI16>);
      else if (I.r <= 32) z0(k_block_z0<32, kCoordI16>);
      else z0(k_block_z0<64, kCoordI16>);
    } else {
      if (I.r <= 8) z0(k_block_z0<8, kCoordF32>);
      else if (I.r <= 16) z0(k_block_z0<16, kCoordF32>);
      else if (I.r <= 32) z0(k_block_z0<32, kCoordF32>);
      else z0(k_block_z0<64, kCoordF32>);
    }
  }
  // Mode A: every id's stored position and h_i = z_i^T G_g z_i of every row
  if (!bf16) k_gram_f32<<<I.G, 256>>>(I.U, (int)I.d, (int)I.r, I.gram);
  HNTL_CUDA_TRY(cudaMemset(I.pos_of_id, 0, sizeof(uint32_t) * std::max<uint64_t>(I.n, 1)));
  if (I.n_blocks) {
    const size_t npos = (size_t)I.n_blocks * kBlockRows;
    k_pos_of_id<<<(unsigned)((npos + 255) / 256), 256>>>(I.ids, npos, I.pos_of_id);
    const Coords cz{I.Zb, I.Z8b, I.scale, I.Z16b};
    const unsigned nb = (unsigned)I.n_blocks;
    const int r = (int)I.r, rp = (int)I.rp;
    if (bf16) {
      if (I.r <= 16) k_row_h<16, kCoordFP8><<<nb, kBlockRows>>>(cz, I.blk_grain, I.gram, r, rp, I.hrow);
      else if (I.r <= 32) k_row_h<32, kCoordFP8><<<nb, kBlockRows>>>(cz, I.blk_grain, I.gram, r, rp, I.hrow);
      else k_row_h<64, kCoordFP8><<<nb, kBlockRows>>>(cz, I.blk_grain, I.gram, r, rp, I.hrow);
    } else if (I.precision == HNTL_PREC_INT16) {
      // no Mode A for the 16-bit form (its query coordinates are replaced by grid values)
    } else {
      if (I.r <= 8) k_row_h<8, kCoordF32><<<nb, kBlockRows>>>(cz, I.blk_grain, I.gram, r, rp, I.hrow);
      else if (I.r <= 16) k_row_h<16, kCoordF32><<<nb, kBlockRows>>>(cz, I.blk_grain, I.gram, r, rp, I.hrow);
      else if (I.r <= 32) k_row_h<32, kCoordF32><<<nb, kBlockRows>>>(cz, I.blk_grain, I.gram, r, rp, I.hrow);
      else k_row_h<64, kCoordF32><<<nb, kBlockRows>>>(cz, I.blk_grain, I.gram, r, rp, I.hrow);
    }
  }
  HNTL_CUDA_TRY(cudaDeviceGetAttribute(&I.num_sms, cudaDevAttrMultiProcessorCount, I.device));
  HNTL_CUDA_TRY(cudaGetLastError());
  HNTL_CUDA_TRY(cudaDeviceSynchronize());
  // tensor-core routing needs 16-byte row strides and the query row in shared memory
  const bool shape_ok = (bf16 ? I.d % 8 == 0 : I.d % 4 == 0) && I.d <= 8192;
  I.tc_route = shape_ok && make_tma_map(&I.mapM, bf16 ? (const void*)I.Mh : (const void*)I.M, bf16, I.G, I.d, kRTN);
  I.tc_proj = bf16 && shape_ok && make_tma_map(&I.mapU, I.Uh, true, (uint64_t)I.G * I.r, I.d, I.r);
  I.tc_proj32 = tc32_shape && make_tma_map(&I.mapU3, I.U3, true, 3ull * I.G * I.r, I.d, I.r);
  return HNTL_OK;
}

}  // namespace hntl

extern "C" {

int hntl_profile_enable(int on) {
  hntl::clear_error();
  hntl::Profiler& P = hntl::profiler();
  std::lock_guard<std::mutex> lk(P.mu);
  P.on = on != 0;
  return HNTL_OK;
}

int hntl_profile_read(double* ms, uint64_t* calls) {
  hntl::clear_error();
  if (!ms || !calls) return hntl::fail(HNTL_EINVAL, "null argument");
  hntl::Profiler& P = hntl::profiler();
  std::lock_guard<std::mutex> lk(P.mu);
  for (int s = 0; s < HNTL_NSTAGES; ++s) ms[s] = 0.0;
  *calls = 0;
  for (auto& ev : P.pending) {
    HNTL_CUDA_TRY(cudaEventSynchronize(ev[HNTL_NSTAGES]));
    for (int s = 0; s < HNTL_NSTAGES; ++s) {
      float t = 0.f;
      HNTL_CUDA_TRY(cudaEventElapsedTime(&t, ev[s], ev[s + 1]));
      ms[s] += t;
    }
    ++*calls;
    P.pool.push_back(ev);
  }
  P.pending.clear();
  return HNTL_OK;
}

int hntl_search_survivors(const hntl_index* idx, const void* d_ws, size_t ws_bytes, uint32_t nq, uint32_t C,
                          uint32_t nprobe, uint32_t* d_counts, void* stream) {
  hntl::clear_error();
  if (!idx || !d_ws || !d_counts) return hntl::fail(HNTL_EINVAL, "null argument");
  uint32_t Ce = C;
  if (hntl::check_params(idx->I, nq, 1, Ce, nprobe)) return HNTL_EINVAL;
  const hntl::Ws w = hntl::carve(idx->I, nq, Ce, nprobe, const_cast<void*>(d_ws));
  if (ws_bytes < w.bytes) return hntl::fail(HNTL_EINVAL, "workspace too small");
  HNTL_CUDA_TRY(cudaMemcpyAsync(d_counts, w.cnt, sizeof(uint32_t) * nq, cudaMemcpyDeviceToDevice,
                                static_cast<cudaStream_t>(stream)));
  return HNTL_OK;
}

size_t hntl_search_workspace_bytes(const hntl_index* idx, uint32_t nq, uint32_t k, uint32_t C, uint32_t nprobe) {
  hntl::clear_error();
  if (!idx) {
    hntl::fail(HNTL_EINVAL, "null index");
    return 0;
  }
  return hntl::workspace_bytes(idx->I, nq, k, C, nprobe);
}

int hntl_search(const hntl_index* idx, const float* d_queries, uint32_t nq, uint32_t k, uint32_t C, uint32_t nprobe,
                const int64_t* d_filter, void* d_ws, size_t ws_bytes, int64_t* d_out_ids, float* d_out_dist,
                uint32_t* d_cand_ids, float* d_cand_dist, int32_t* d_probe, void* stream) {
  hntl::clear_error();
  if (!idx) return hntl::fail(HNTL_EINVAL, "null index");
  return hntl::search(idx->I, d_queries, nq, k, C, nprobe, d_filter, d_ws, ws_bytes, d_out_ids, d_out_dist,
                      d_cand_ids, d_cand_dist, d_probe, static_cast<cudaStream_t>(stream));
}

int hntl_search_mode_a(const hntl_index* idx, const float* d_queries, uint32_t nq, uint32_t k, uint32_t C,
                       uint32_t nprobe, const int64_t* d_filter, void* d_ws, size_t ws_bytes, int64_t* d_out_ids,
                       float* d_out_dist, uint32_t* d_cand_ids, float* d_cand_dist, void* stream) {
  hntl::clear_error();
  if (!idx) return hntl::fail(HNTL_EINVAL, "null index");
  return hntl::search(idx->I, d_queries, nq, k, C, nprobe, d_filter, d_ws, ws_bytes, d_out_ids, d_out_dist,
                      d_cand_ids, d_cand_dist, nullptr, static_cast<cudaStream_t>(stream), nullptr, nullptr,
                      nullptr, true);
}

int hntl_search_probes(const hntl_index* idx, const float* d_queries, uint32_t nq, uint32_t k, uint32_t C,
                       uint32_t nprobe, const int32_t* d_probe_in, const int64_t* d_filter, void* d_ws,
                       size_t ws_bytes, int64_t* d_out_ids, float* d_out_dist, uint32_t* d_cand_ids,
                       float* d_cand_dist, void* stream) {
  hntl::clear_error();
  if (!idx) return hntl::fail(HNTL_EINVAL, "null index");
  if (!d_probe_in && nq) return hntl::fail(HNTL_EINVAL, "null probe list");
  return hntl::search(idx->I, d_queries, nq, k, C, nprobe, d_filter, d_ws, ws_bytes, d_out_ids, d_out_dist,
                      d_cand_ids, d_cand_dist, nullptr, static_cast<cudaStream_t>(stream), d_probe_in);
}

int hntl_search_pair_codes(const hntl_index* idx, const void* d_ws, size_t ws_bytes, uint32_t nq, uint32_t C,
                           uint32_t nprobe, int16_t* d_codes, int32_t* d_rcodes, void* stream) {
  hntl::clear_error();
  if (!idx || !d_ws || !d_codes || !d_rcodes) return hntl::fail(HNTL_EINVAL, "null argument");
  const hntl::Index& I = idx->I;
  if (I.precision != HNTL_PREC_INT16) return hntl::fail(HNTL_EINVAL, "query codes exist in the 16-bit form only");
  uint32_t Ce = C;
  if (hntl::check_params(I, nq, 1, Ce, nprobe)) return HNTL_EINVAL;
  const hntl::Ws w = hntl::carve(I, nq, Ce, nprobe, const_cast<void*>(d_ws));
  if (ws_bytes < w.bytes) return hntl::fail(HNTL_EINVAL, "workspace too small");
  const uint32_t n = nq * nprobe;
  if (n == 0) return HNTL_OK;
  hntl::DeviceGuard dg(I.device);
  hntl::k_gather_pair_codes<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n, (int)I.r, (int)I.rp, w.pair_of, w.zq16, w.rc16, d_codes, d_rcodes);
  HNTL_CUDA_TRY(cudaGetLastError());
  return HNTL_OK;
}

namespace hntl {
namespace {
// Diagnostic gather of each pair's projection into query order: z_q [n][r] and rho_q [n].
__global__ void k_gather_pair_proj(uint32_t n, int r, const uint32_t* __restrict__ pair_of,
                                   const float* __restrict__ zq, const float* __restrict__ rhoq,
                                   float* __restrict__ z_out, float* __restrict__ rho_out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t pr = pair_of[i];
  for (int j = 0; j < r; ++j) z_out[(size_t)i * r + j] = zq[(size_t)pr * r + j];
  rho_out[i] = rhoq[pr];
}
}  // namespace
}  // namespace hntl

int hntl_search_pair_proj(const hntl_index* idx, const void* d_ws, size_t ws_bytes, uint32_t nq, uint32_t C,
                          uint32_t nprobe, float* d_zq, float* d_rhoq, void* stream) {
  hntl::clear_error();
  if (!idx || !d_ws || !d_zq || !d_rhoq) return hntl::fail(HNTL_EINVAL, "null argument");
  const hntl::Index& I = idx->I;
  uint32_t Ce = C;
  if (hntl::check_params(I, nq, 1, Ce, nprobe)) return HNTL_EINVAL;
  const hntl::Ws w = hntl::carve(I, nq, Ce, nprobe, const_cast<void*>(d_ws));
  if (ws_bytes < w.bytes) return hntl::fail(HNTL_EINVAL, "workspace too small");
  const uint32_t n = nq * nprobe;
  if (n == 0) return HNTL_OK;
  hntl::DeviceGuard dg(I.device);
  hntl::k_gather_pair_proj<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      n, (int)I.r, w.pair_of, w.zq, w.rhoq, d_zq, d_rhoq);
  HNTL_CUDA_TRY(cudaGetLastError());
  return HNTL_OK;
}

int hntl_debug_set_persistent_cap(uint32_t ctas) {
  hntl::clear_error();
  hntl::g_persistent_cap.store(ctas, std::memory_order_relaxed);
  return HNTL_OK;
}

int hntl_search_scan_stats(const hntl_index* idx, const void* d_ws, size_t ws_bytes, uint32_t nq, uint32_t C,
                           uint32_t nprobe, uint32_t* d_stats, void* stream) {
  hntl::clear_error();
  if (!idx || !d_ws || !d_stats) return hntl::fail(HNTL_EINVAL, "null argument");
  uint32_t Ce = C;
  if (hntl::check_params(idx->I, nq, 1, Ce, nprobe)) return HNTL_EINVAL;
  const hntl::Ws w = hntl::carve(idx->I, nq, Ce, nprobe, const_cast<void*>(d_ws));
  if (ws_bytes < w.bytes) return hntl::fail(HNTL_EINVAL, "workspace too small");
  HNTL_CUDA_TRY(cudaMemcpyAsync(d_stats, w.cnt + nq, sizeof(uint32_t) * 5, cudaMemcpyDeviceToDevice,
                                static_cast<cudaStream_t>(stream)));
  return HNTL_OK;
}

int hntl_selftest_wait_timeout(const hntl_index* idx, uint32_t polls, void* stream) {
  hntl::clear_error();
  if (!idx || polls == 0 || polls > (1u << 20)) return hntl::fail(HNTL_EINVAL, "polls must be in [1, 2^20]");
  hntl::k_wait_selftest<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(polls, idx->I.d_err);
  HNTL_CUDA_TRY(cudaGetLastError());
  return HNTL_OK;
}

int hntl_device_status(const hntl_index* idx, int* status, int clear) {
  hntl::clear_error();
  if (!idx || !status) return hntl::fail(HNTL_EINVAL, "null argument");
  const hntl::Index& I = idx->I;
  HNTL_CUDA_TRY(cudaMemcpy(status, I.d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (clear) HNTL_CUDA_TRY(cudaMemset(I.d_err, 0, sizeof(int)));
  return (*status & 1) ? HNTL_ETIMEOUT : HNTL_OK;
}

int hntl_route(const hntl_index* idx, const float* d_queries, uint32_t nq, uint32_t nprobe, void* d_ws,
               size_t ws_bytes, int32_t* d_probe, float* d_probe_dist, void* stream) {
  hntl::clear_error();
  if (!idx) return hntl::fail(HNTL_EINVAL, "null index");
  return hntl::route_only(idx->I, d_queries, nq, nprobe, d_ws, ws_bytes, d_probe, d_probe_dist,
                          static_cast<cudaStream_t>(stream));
}

size_t hntl_search_host_workspace_bytes(const hntl_index* idx, uint32_t nq, uint32_t k, uint32_t C, uint32_t nprobe,
                                        int with_filter) {
  hntl::clear_error();
  if (!idx) {
    hntl::fail(HNTL_EINVAL, "null index");
    return 0;
  }
  size_t need = hntl::workspace_bytes(idx->I, nq, k, C, nprobe);
  if (need == 0) return 0;
  hntl::Carver c(nullptr);
  c.take<float>((size_t)nq * idx->I.d);
  if (with_filter) c.take<int64_t>((size_t)nq * 2);
  c.take<int64_t>((size_t)nq * k);
  c.take<float>((size_t)nq * k);
  return need + hntl::align_up(c.off, 256);
}

int hntl_search_host(const hntl_index* idx, const float* h_queries, uint32_t nq, uint32_t k, uint32_t C,
                     uint32_t nprobe, const int64_t* h_filter, void* d_ws, size_t ws_bytes, int64_t* h_out_ids,
                     float* h_out_dist, void* stream) {
  hntl::clear_error();
  if (!idx) return hntl::fail(HNTL_EINVAL, "null index");
  const hntl::Index& I = idx->I;
  if (nq == 0) return HNTL_OK;
  if (!h_queries || !h_out_ids || !h_out_dist || !d_ws) return hntl::fail(HNTL_EINVAL, "null buffer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // device staging for queries, filters and results follows the search workspace
  size_t need = hntl::workspace_bytes(I, nq, k, C, nprobe);
  if (need == 0) return HNTL_EINVAL;
  hntl::Carver c(static_cast<char*>(d_ws) + need);
  float* dQ = c.take<float>((size_t)nq * I.d);
  int64_t* dF = h_filter ? c.take<int64_t>((size_t)nq * 2) : nullptr;
  int64_t* dI = c.take<int64_t>((size_t)nq * k);
  float* dD = c.take<float>((size_t)nq * k);
  size_t total = need + hntl::align_up(c.off, 256);
  if (ws_bytes < total) return hntl::fail(HNTL_EINVAL, "workspace too small for the host form");
  HNTL_CUDA_TRY(cudaMemcpyAsync(dQ, h_queries, sizeof(float) * nq * I.d, cudaMemcpyHostToDevice, st));
  if (dF) HNTL_CUDA_TRY(cudaMemcpyAsync(dF, h_filter, sizeof(int64_t) * nq * 2, cudaMemcpyHostToDevice, st));
  int rc = hntl::search(I, dQ, nq, k, C, nprobe, dF, d_ws, need, dI, dD, nullptr, nullptr, nullptr, st);
  if (rc) return rc;
  HNTL_CUDA_TRY(cudaMemcpyAsync(h_out_ids, dI, sizeof(int64_t) * nq * k, cudaMemcpyDeviceToHost, st));
  HNTL_CUDA_TRY(cudaMemcpyAsync(h_out_dist, dD, sizeof(float) * nq * k, cudaMemcpyDeviceToHost, st));
  HNTL_CUDA_TRY(cudaStreamSynchronize(st));
  return HNTL_OK;
}

}  // extern "C"
