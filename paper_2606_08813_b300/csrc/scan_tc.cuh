// Block-SoA scan of the precision form on the tensor cores (Eq. 6, with the
// pool filter of the fused scan).
//
// For a probed grain g, every (row i, pair p) needs D = ||z_q - z_i||^2 +
// rho_q + rho_i. Expanded, D = (||z_q||^2 + rho_q) + (||z_i||^2 + rho_i)
// - 2 z_q . z_i, and the cross terms of a 128-row block against the grain's
// pairs are one small dense contraction, K = r:
//   A = the block's FP8-E4M3 codes, converted exactly to FP16 (128 x rp),
//   B = each pair's z_q scaled by a power of two sigma_p (so that its largest
//       coordinate is in [2^13, 2^14)) and split into FP16 hi + lo parts,
//   z_q . z_i = s_g / sigma_p * (code_i . (hi_p + lo_p)), FP32 accumulation.
// The expansion is only used to discard rows: with c_i = ||z_i||^2 + rho_i
// precomputed per row and A_p = ||z_q||^2 + rho_q,
//   |D~ - D| <= 2^-14 (A_p + c_i)
// bounds every error of the approximate D~ (the hi/lo split keeps 22 bits of
// z_q, each FP16 product is exact in FP32, the accumulation over 2 rp terms
// is charged 2^-16 of sum |products| <= ||z_q|| ||z_i||, the rest are a few
// FP32 roundings of magnitude <= A_p + c_i), so a row whose D~ minus that
// margin exceeds tau_p cannot survive. The few rows that pass are evaluated
// with eval_D, exactly as in the SIMT scan, and kept when D <= tau_p and the
// attribute is in range: the survivor set is the same set of (D, id) keys.
//
// Persistent CTAs take work items (a probed grain, up to 8 of its consecutive
// blocks) from a global counter, so grains probed by many queries (hubs, in
// high dimension) spread over the CTAs. An item first keeps the pairs that can
// reach their pool from one of its blocks (rho_q + min rho_block <= tau_q, as
// D >= rho_q + rho_i). After that pruning most items of clustered data keep
// one or two pairs, which is no contraction: an item with fewer than
// kSTDense live pairs evaluates them row by row in the direct form. Denser
// items, per round of up to 128 pairs, build the B operand (one thread per
// pair), and blocks then flow through a two-deep pipeline:
// convert block i
// into A[i % 2], issue its MMAs into TMEM accumulator i % 2, and run the
// epilogue of block i - 1 while they execute. Per row the scan streams only
// the codes and c_i (rp + 4 bytes); ids, rho and attributes are read for
// candidates only.
#pragma once

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "hntl_internal.cuh"
#include "project_tc.cuh"  // sw128_off
#include "scan_select.cuh"
#include "tc_common.cuh"

namespace hntl {
namespace {

constexpr int kSTBlocks = 8;    // blocks per work item (consecutive blocks of one grain)
constexpr int kSTNeed = 1024;   // pairs of a grain one item can list after pruning
constexpr int kSTDense = 8;     // from this many live pairs an item contracts on the tensor cores
constexpr int kSTN = 128;       // pairs per round (MMA N <= 128)
constexpr int kSTThreads = 128;  // thread t = row t = TMEM lane t

// Two E4M3 codes (low byte first) to two FP16 values (low half first); exact.
__device__ __forceinline__ uint32_t fp8x2_to_half2_bits(uint32_t w16) {
  const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)w16, __NV_E4M3);
  return (uint32_t)h.x | ((uint32_t)h.y << 16);
}

template <int RT>
struct ScanTc {
  static constexpr uint32_t kBytesA = kBlockRows * 128;  // SW128 rows; rp * 2 bytes of each are used
  static constexpr uint32_t kBytesB = kSTN * 128;
  static constexpr int kSmem = 2 * kBytesA + 2 * kBytesB + kSTN * RT * 4 + 1024;
};

// Smallest residual norm of each grain's rows (+inf for an empty grain), one warp per grain.
__global__ void k_grain_rho_min(const float* __restrict__ blk_rho_min, const uint32_t* __restrict__ blk_off, int G,
                                float* __restrict__ out) {
  const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (g >= G) return;
  float v = INFINITY;
  for (uint32_t b = blk_off[g] + lane; b < blk_off[g + 1]; b += 32) v = fminf(v, blk_rho_min[b]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) out[g] = v;
}

// c_i = ||z_i||^2 + rho_i of every row, z_i decoded exactly as the scan decodes it.
template <int RT>
__global__ void __launch_bounds__(kBlockRows) k_row_c(const Coords cz, const float* __restrict__ rho,
                                                      const uint32_t* __restrict__ blk_grain, int rp,
                                                      float* __restrict__ c_out) {
  const size_t b = blockIdx.x;
  const int t = threadIdx.x;
  float z[RT];
  load_row<RT, true>(cz, rp, cz.scale[blk_grain[b]], b, t, z);
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < RT; ++j) s = fmaf(z[j], z[j], s);
  c_out[b * kBlockRows + t] = s + rho[b * kBlockRows + t];
}

// Per probed grain, the pairs that can reach their pool from some row of the
// grain at all (rho_q + min rho over the grain <= tau_q, as D >= rho_q +
// rho_i): their indices within the grain's pair list, compacted at the
// grain's pair offset, and their number. One CTA per grain.
__global__ void __launch_bounds__(128) k_grain_needed(const uint32_t* __restrict__ gcnt,
                                                      const uint32_t* __restrict__ pair_off,
                                                      const uint32_t* __restrict__ pair_q,
                                                      const float* __restrict__ rhoq, const float* __restrict__ tau,
                                                      const float* __restrict__ grain_rho_min,
                                                      uint32_t* __restrict__ need_list,
                                                      uint32_t* __restrict__ need_cnt) {
  __shared__ uint32_t s_n;
  const uint32_t g = blockIdx.x, m = gcnt[g], p0 = pair_off[g];
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  const float rmin = grain_rho_min[g];
  for (uint32_t s = threadIdx.x; s < m; s += blockDim.x) {
    if (rhoq[p0 + s] + rmin <= tau[pair_q[p0 + s]]) need_list[p0 + atomicAdd(&s_n, 1u)] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) need_cnt[g] = s_n;
}

// A sparse work item as the classifier leaves it: the item and the pairs
// (indices into the batch's pair arrays) live in it.
struct SparseRec {
  uint4 item;                    // grain, first block, blocks, live pairs
  uint32_t pr[kSTDense - 1];     // live pairs
  uint32_t pad;
};

// Sorts the scan's work items by how many of their grain's live pairs can
// still reach their pool from the item's blocks (rho_q + min rho_block <=
// tau_q): none (dropped), a few (recorded with those pairs for the
// direct-form kernel), at least kSTDense (the tensor-core kernel). One warp
// per item. lists: [0] dense count, [1] light sparse count, [3] heavy sparse
// count. Sparse records of light items fill the buffer (n_cap records) from
// the front and those of heavy items (blocks x (1 + live pairs) >= 24) from
// the back, so the scan can take the costly items first and finish on short
// ones.
__global__ void k_scan_classify(const uint4* __restrict__ items, const uint32_t* __restrict__ n_items,
                                const uint32_t* __restrict__ need_cnt, const uint32_t* __restrict__ need_list,
                                const uint32_t* __restrict__ pair_off, const uint32_t* __restrict__ pair_q,
                                const float* __restrict__ rhoq, const float* __restrict__ tau,
                                const float* __restrict__ blk_rho_min, const float2* __restrict__ blk_z0,
                                const float* __restrict__ zq, int r, uint4* __restrict__ dense,
                                SparseRec* __restrict__ sparse, uint32_t n_cap, uint32_t* __restrict__ lists) {
  const uint32_t w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= *n_items) return;
  const uint4 item = items[w];
  float v = (uint32_t)lane < item.z ? blk_rho_min[item.y + lane] : INFINITY;
  float2 iv = (uint32_t)lane < item.z ? blk_z0[item.y + lane] : make_float2(INFINITY, -INFINITY);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    iv.x = fminf(iv.x, __shfl_xor_sync(0xffffffffu, iv.x, o));
    iv.y = fmaxf(iv.y, __shfl_xor_sync(0xffffffffu, iv.y, o));
  }
  const uint32_t m = need_cnt[item.x], p0 = pair_off[item.x];
  uint32_t n = 0, mine = 0xFFFFFFFFu;  // lane i < n keeps the i-th live pair
  for (uint32_t s0 = 0; s0 < m && n < (uint32_t)kSTDense; s0 += 32) {
    const uint32_t s = s0 + lane;
    bool need = false;
    uint32_t pr = 0;
    if (s < m) {
      pr = p0 + need_list[p0 + s];
      const float rq = rhoq[pr], tq = tau[pair_q[pr]];
      need = rq + v <= tq && !interval_prunes(zq[(size_t)pr * r], iv, rq, v, tq);
    }
    const unsigned mask = __ballot_sync(0xffffffffu, need);
    const uint32_t slot = n + __popc(mask & ((1u << lane) - 1u));
    // hand the pair to lane `slot` (one pass: each live pair has a distinct slot)
    for (int src = 0; src < 32; ++src) {
      const uint32_t p_src = __shfl_sync(0xffffffffu, pr, src);
      const uint32_t slot_src = __shfl_sync(0xffffffffu, slot, src);
      if (((mask >> src) & 1u) && slot_src == (uint32_t)lane) mine = p_src;
    }
    n += __popc(mask);
  }
  if (!n) return;
  if (n >= (uint32_t)kSTDense) {
    if (lane == 0) dense[atomicAdd(&lists[0], 1u)] = item;
    return;
  }
  uint32_t pos = 0;
  if (lane == 0)
    pos = item.z * (1u + n) >= 24u ? n_cap - 1u - atomicAdd(&lists[3], 1u) : atomicAdd(&lists[1], 1u);
  pos = __shfl_sync(0xffffffffu, pos, 0);
  if (lane == 0) sparse[pos].item = make_uint4(item.x, item.y, item.z, n);
  if ((uint32_t)lane < n) sparse[pos].pr[lane] = mine;
}

constexpr int kSPThreads = 128;

// Direct-form scan of the items with fewer than kSTDense live pairs: one row
// per thread, the item's blocks streamed with two blocks of codes prefetched
// in registers, each live pair evaluated by eval_D (the same function, on the
// same decoded coordinates, as the pilot and the pool fallback).
template <int RT>
__global__ void __launch_bounds__(kSPThreads, 6) k_scan_sparse(
    const SparseRec* __restrict__ recs, uint32_t n_cap, const uint32_t* __restrict__ lists,
    uint32_t* __restrict__ next_item,
    const uint32_t* __restrict__ blk_off,
    const uint32_t* __restrict__ grain_rows, const uint8_t* __restrict__ Z8b, const float* __restrict__ scale,
    const float* __restrict__ rho, const uint32_t* __restrict__ ids, const int64_t* __restrict__ attr_b, int r,
    int rp, const uint32_t* __restrict__ pair_q, const float* __restrict__ zq, const float* __restrict__ rhoq,
    const float* __restrict__ tau, const float* __restrict__ blk_rho_min, const float2* __restrict__ blk_z0,
    const int64_t* __restrict__ filter, uint32_t cap, uint32_t* __restrict__ cnt,
    unsigned long long* __restrict__ surv) {
  constexpr int kL = RT / 16;
  constexpr int kP = kSTDense - 1;  // at most this many live pairs per item
  __shared__ __align__(16) float sz[kP][RT];
  __shared__ float4 spc[kP];  // {unused, unused, tau_q, rho_q}
  __shared__ uint32_t sqid[kP], spr[kP];
  __shared__ long long slo[kP], shi[kP];
  const int t = threadIdx.x, lane = t & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const uint32_t heavy = lists[3], total = lists[1] + heavy;  // heavy items (at the back) first
  const int nks = rp / 16;
  // items taken from a global counter (their costs vary; a static split left a
  // tail); the next item's index is claimed while the current one is scanned
  __shared__ uint32_t s_item;
  if (t == 0) s_item = atomicAdd(next_item, 1u);
  __syncthreads();
  uint32_t w = s_item;
  while (w < total) {
    const SparseRec& rec = recs[w < heavy ? n_cap - 1u - w : w - heavy];
    const uint4 item = rec.item;
    const uint32_t my_pr = t < kP ? rec.pr[t] : 0u;
    const uint32_t g = item.x, b0 = item.y, nb = item.z;
    const int np = (int)item.w;
    const uint32_t n_g = grain_rows[g], gb0 = blk_off[g];
    const float s_g = scale[g];
    uint4 cur[kL], nxt[kL];
    float rho_cur = 0.f, rho_nxt = 0.f, rmin_cur = 0.f, rmin_nxt = 0.f;
    auto load_block = [&](uint32_t i, uint4 (&codes)[kL], float& rh, float& rmin) {
      const size_t b = b0 + i;
#pragma unroll
      for (int l = 0; l < kL; ++l)
        if (l < nks)
          codes[l] = __ldg(reinterpret_cast<const uint4*>(Z8b + ((b * (size_t)nks + l) * kBlockRows + t) * 16));
      rh = rho[b * kBlockRows + t];
      rmin = blk_rho_min[b];
    };
    load_block(0, cur, rho_cur, rmin_cur);
    if (nb > 1) load_block(1, nxt, rho_nxt, rmin_nxt);
    __syncthreads();  // every thread is done with the previous item's pair data
    if (t < np) spr[t] = my_pr;  // threads 0..kP-1 hold the item's pairs
    __syncthreads();
    for (int e = t; e < np * RT; e += kSPThreads) {
      const int j = e / RT, a = e % RT;
      sz[j][a] = a < r ? zq[(size_t)spr[j] * r + a] : 0.f;
    }
    if (t < np) {
      const uint32_t q = pair_q[my_pr];
      spc[t] = make_float4(0.f, 0.f, tau[q], rhoq[my_pr]);
      sqid[t] = q;
      if (filter) {
        slo[t] = (long long)filter[2 * (size_t)q];
        shi[t] = (long long)filter[2 * (size_t)q + 1];
      }
    }
    if (t == 0) s_item = atomicAdd(next_item, 1u);  // read after the barrier below
    __syncthreads();
    w = s_item;
    for (uint32_t i = 0; i < nb; ++i) {
      const size_t b = b0 + i;
      const bool valid = (uint32_t)(b - gb0) * kBlockRows + t < n_g;
      float z[RT];
#pragma unroll
      for (int l = 0; l < kL; ++l) {
        if (l < nks) {
          const uint32_t wv[4] = {cur[l].x, cur[l].y, cur[l].z, cur[l].w};
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const float2 a2 = __half22float2(
                __half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(wv[h] & 0xFFFFu), __NV_E4M3)));
            const float2 e2 = __half22float2(
                __half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(wv[h] >> 16), __NV_E4M3)));
            z[l * 16 + 4 * h + 0] = a2.x * s_g;
            z[l * 16 + 4 * h + 1] = a2.y * s_g;
            z[l * 16 + 4 * h + 2] = e2.x * s_g;
            z[l * 16 + 4 * h + 3] = e2.y * s_g;
          }
        } else {
#pragma unroll
          for (int k = 0; k < 16; ++k) z[l * 16 + k] = 0.f;
        }
      }
      const float rho_i = rho_cur, rmin = rmin_cur;
      const float2 iv = blk_z0[b];
      for (int j = 0; j < np; ++j) {
        const float4 pc = spc[j];
        // block-uniform: no row of this block reaches the pool
        if (pc.w + rmin > pc.z || interval_prunes(sz[j][0], iv, pc.w, rmin, pc.z)) continue;
        const float D = eval_D<RT>(&sz[j][0], z, pc.w, rho_i);
        bool ok = valid && D <= pc.z;
        if (ok && filter) {
          const long long av = (long long)attr_b[b * kBlockRows + t];
          ok = av >= slo[j] && av <= shi[j];
        }
        const unsigned mask = __ballot_sync(0xffffffffu, ok);
        if (mask) {
          const int leader = __ffs(mask) - 1;
          uint32_t base = 0;
          if (lane == leader) base = atomicAdd(&cnt[sqid[j]], (uint32_t)__popc(mask));
          base = __shfl_sync(0xffffffffu, base, leader);
          if (ok) {
            const uint32_t pos = base + __popc(mask & lt_mask);
            if (pos < cap)
              surv[(size_t)sqid[j] * cap + pos] = ((unsigned long long)__float_as_uint(D) << 32) | ids[b * kBlockRows + t];
          }
        }
      }
#pragma unroll
      for (int l = 0; l < kL; ++l) cur[l] = nxt[l];
      rho_cur = rho_nxt;
      rmin_cur = rmin_nxt;
      if (i + 2 < nb) load_block(i + 2, nxt, rho_nxt, rmin_nxt);
    }
  }
}

template <int RT>
__global__ void __launch_bounds__(kSTThreads, 2) k_scan_tc(
    const uint4* __restrict__ items, const uint32_t* __restrict__ n_items, uint32_t* __restrict__ next_item,
    const uint32_t* __restrict__ blk_off, const uint32_t* __restrict__ grain_rows, const uint8_t* __restrict__ Z8b,
    const float* __restrict__ scale, const float* __restrict__ crow, const float* __restrict__ rho,
    const uint32_t* __restrict__ ids, const int64_t* __restrict__ attr_b, int r, int rp,
    const uint32_t* __restrict__ need_cnt, const uint32_t* __restrict__ need_list,
    const uint32_t* __restrict__ pair_off, const uint32_t* __restrict__ pair_q,
    const float* __restrict__ zq, const float* __restrict__ rhoq, const float* __restrict__ tau,
    const float* __restrict__ blk_rho_min, const int64_t* __restrict__ filter, uint32_t cap,
    uint32_t* __restrict__ cnt, unsigned long long* __restrict__ surv, int* __restrict__ err) {
  using P = ScanTc<RT>;
  constexpr int kL = RT / 16;  // 16-code lanes per row (at most)
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;                                        // [2][kBytesA]
  uint8_t* sBh = smem + 2 * P::kBytesA;                      // [kBytesB]
  uint8_t* sBl = sBh + P::kBytesB;                           // [kBytesB]
  float* sz = reinterpret_cast<float*>(sBl + P::kBytesB);    // [kSTN][RT] z_q (FP32, zero padded)
  __shared__ float4 spc[kSTN];  // per pair: {A_p (1 - 2^-14), 2 s_g / sigma_p, tau_q, rho_q}
  __shared__ uint32_t sqid[kSTN];
  __shared__ long long slo[kSTN], shi[kSTN];
  __shared__ uint32_t s_need[kSTNeed];
  __shared__ uint32_t s_nneed, s_item;
  __shared__ float s_rmin;
  __shared__ __align__(8) uint64_t mbar[2], fin;
  __shared__ uint32_t tmem_base;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  if (warp == 0) tc::tmem_alloc(&tmem_base, 2 * kSTN);
  if (t == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_init(&fin, 1);
    tc::mbar_fence_init();
  }
  bool issued = false;  // thread 0: has this CTA issued MMAs
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t total = *n_items;
  const int nks = rp / 16;
  uint32_t ph = 0u;  // bit e: phase of accumulator e's barrier
  bool failed = false;
  const unsigned lt_mask = (1u << lane) - 1u;

  for (;;) {
    __syncthreads();  // every thread is done with the previous item
    if (t == 0) s_item = atomicAdd(next_item, 1u);
    __syncthreads();
    const uint32_t w = s_item;
    if (w >= total || failed) break;
    const uint4 item = items[w];
    const uint32_t g = item.x, b0 = item.y, nb = item.z;
    const uint32_t m = need_cnt[g], p_begin = pair_off[g], n_g = grain_rows[g], gb0 = blk_off[g];
    const float s_g = scale[g];
    // pairs that can reach their pool from some block of this item (D >= rho_q + rho_i)
    if (warp == 0) {
      float v = (uint32_t)lane < nb ? blk_rho_min[b0 + lane] : INFINITY;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (lane == 0) {
        s_rmin = v;
        s_nneed = 0;
      }
    }
    __syncthreads();
    const float rmin_item = s_rmin;
    for (uint32_t i = t; i < m; i += kSTThreads) {
      const uint32_t sidx = need_list[p_begin + i];
      const uint32_t pr = p_begin + sidx;
      if (rhoq[pr] + rmin_item <= tau[pair_q[pr]]) {
        const uint32_t pos = atomicAdd(&s_nneed, 1u);
        if (pos < (uint32_t)kSTNeed) s_need[pos] = sidx;
      }
    }
    __syncthreads();
    const uint32_t nneed = s_nneed;
    const bool listed = nneed <= (uint32_t)kSTNeed;  // else walk every live pair of the grain
    const uint32_t nwalk = listed ? nneed : m;
    for (uint32_t s0 = 0; s0 < nwalk && !failed; s0 += kSTN) {
      const int np = (int)min((uint32_t)kSTN, nwalk - s0);
      const int N = (np + 15) & ~15;
      __syncthreads();  // every thread is done with the previous round's pair data
      // ---- B operand and per-pair constants, one thread per pair
      if (t < np) {
        const uint32_t pr = p_begin + (listed ? s_need[s0 + t] : need_list[p_begin + s0 + t]);
        float zv[RT];
#pragma unroll
        for (int a = 0; a < RT; ++a) zv[a] = a < r ? zq[(size_t)pr * r + a] : 0.f;
        float mx = 0.f, nn = 0.f;
#pragma unroll
        for (int a = 0; a < RT; ++a) {
          mx = fmaxf(mx, fabsf(zv[a]));
          nn = fmaf(zv[a], zv[a], nn);
        }
        // sigma = 2^(13 - e), e = exponent of the largest coordinate (clamped)
        int e = (mx > 0.f) ? (int)((__float_as_uint(mx) >> 23) & 0xFF) - 127 : 0;
        e = max(-100, min(100, e));
        const float sigma = __uint_as_float((uint32_t)(127 + 13 - e) << 23);
#pragma unroll
        for (int a0 = 0; a0 < RT; a0 += 8) {
          if (a0 < rp) {
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const float x0 = zv[a0 + 2 * h] * sigma, x1 = zv[a0 + 2 * h + 1] * sigma;
              const __half h0 = __float2half_rn(x0), h1 = __float2half_rn(x1);
              const __half l0 = __float2half_rn(x0 - __half2float(h0)), l1 = __float2half_rn(x1 - __half2float(h1));
              hw[h] = (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
              lw[h] = (uint32_t)__half_as_ushort(l0) | ((uint32_t)__half_as_ushort(l1) << 16);
            }
            const uint32_t off = sw128_off(t, 2 * a0);
            *reinterpret_cast<uint4*>(sBh + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4*>(sBl + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
          }
        }
#pragma unroll
        for (int a = 0; a < RT; a += 4)
          *reinterpret_cast<float4*>(sz + t * RT + a) = make_float4(zv[a], zv[a + 1], zv[a + 2], zv[a + 3]);
        const uint32_t q = pair_q[pr];
        const float rq = rhoq[pr];
        spc[t] = make_float4((nn + rq) * (1.f - 1.f / 16384.f), 2.f * s_g / sigma, tau[q], rq);
        sqid[t] = q;
        if (filter) {
          slo[t] = (long long)filter[2 * (size_t)q];
          shi[t] = (long long)filter[2 * (size_t)q + 1];
        }
      }
      tc::fence_proxy_async_smem();
      const uint32_t idesc = tc::idesc_f32acc(0u, kBlockRows, N);  // FP16 x FP16 -> FP32, 128 x N
      // ---- blocks: convert i, MMA i, epilogue i - 1
      uint4 cur[kL], nxt[kL];
      float c_cur = 0.f, c_nxt = 0.f, c_prev = 0.f;
      float rmin_cur = 0.f, rmin_nxt = 0.f, rmin_prev = 0.f;
      const bool dense = np >= kSTDense;
      auto load_block = [&](uint32_t i, uint4 (&codes)[kL], float& c, float& rmin) {
        const size_t b = b0 + i;
#pragma unroll
        for (int l = 0; l < kL; ++l)
          if (l < nks)
            codes[l] = __ldg(reinterpret_cast<const uint4*>(Z8b + ((b * (size_t)nks + l) * kBlockRows + t) * 16));
        c = dense ? crow[b * kBlockRows + t] : rho[b * kBlockRows + t];  // c_i, or rho_i for the direct path
        rmin = blk_rho_min[b];
      };
      load_block(0, cur, c_cur, rmin_cur);
      if (nb > 1) load_block(1, nxt, c_nxt, rmin_nxt);
      if (!dense) {
        // ---- few live pairs: each thread evaluates its row against them directly (the
        // same eval_D on the same decoded coordinates as the pilot and the fallback)
        __syncthreads();  // pair data written
        for (uint32_t i = 0; i < nb; ++i) {
          const size_t b = b0 + i;
          const bool valid = (uint32_t)(b - gb0) * kBlockRows + t < n_g;
          float z[RT];
#pragma unroll
          for (int l = 0; l < kL; ++l) {
            if (l < nks) {
              const uint32_t wv[4] = {cur[l].x, cur[l].y, cur[l].z, cur[l].w};
#pragma unroll
              for (int h = 0; h < 4; ++h) {
                const float2 a2 = __half22float2(
                    __half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(wv[h] & 0xFFFFu), __NV_E4M3)));
                const float2 e2 = __half22float2(
                    __half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(wv[h] >> 16), __NV_E4M3)));
                z[l * 16 + 4 * h + 0] = a2.x * s_g;
                z[l * 16 + 4 * h + 1] = a2.y * s_g;
                z[l * 16 + 4 * h + 2] = e2.x * s_g;
                z[l * 16 + 4 * h + 3] = e2.y * s_g;
              }
            } else {
#pragma unroll
              for (int k = 0; k < 16; ++k) z[l * 16 + k] = 0.f;
            }
          }
          const float rho_i = c_cur, rmin = rmin_cur;
          for (int j = 0; j < np; ++j) {
            const float4 pc = spc[j];
            if (pc.w + rmin > pc.z) continue;  // block-uniform: no row of this block reaches the pool
            const float D = eval_D<RT>(sz + j * RT, z, pc.w, rho_i);
            bool ok = valid && D <= pc.z;
            if (ok && filter) {
              const long long av = (long long)attr_b[b * kBlockRows + t];
              ok = av >= slo[j] && av <= shi[j];
            }
            const unsigned mask = __ballot_sync(0xffffffffu, ok);
            if (mask) {
              const int leader = __ffs(mask) - 1;
              uint32_t base = 0;
              if (lane == leader) base = atomicAdd(&cnt[sqid[j]], (uint32_t)__popc(mask));
              base = __shfl_sync(0xffffffffu, base, leader);
              if (ok) {
                const uint32_t pos = base + __popc(mask & lt_mask);
                if (pos < cap)
                  surv[(size_t)sqid[j] * cap + pos] =
                      ((unsigned long long)__float_as_uint(D) << 32) | ids[b * kBlockRows + t];
              }
            }
          }
#pragma unroll
          for (int l = 0; l < kL; ++l) cur[l] = nxt[l];
          c_cur = c_nxt;
          rmin_cur = rmin_nxt;
          if (i + 2 < nb) load_block(i + 2, nxt, c_nxt, rmin_nxt);
        }
        continue;
      }
      for (uint32_t i = 0; i <= nb; ++i) {
        if (i < nb) {
          uint8_t* a = sA + (i & 1) * P::kBytesA;
#pragma unroll
          for (int l = 0; l < kL; ++l) {
            if (l < nks) {
              const uint32_t wv[4] = {cur[l].x, cur[l].y, cur[l].z, cur[l].w};
              uint32_t hv[8];
#pragma unroll
              for (int h = 0; h < 4; ++h) {
                hv[2 * h] = fp8x2_to_half2_bits(wv[h] & 0xFFFFu);
                hv[2 * h + 1] = fp8x2_to_half2_bits(wv[h] >> 16);
              }
              *reinterpret_cast<uint4*>(a + sw128_off(t, 32 * l)) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
              *reinterpret_cast<uint4*>(a + sw128_off(t, 32 * l + 16)) = make_uint4(hv[4], hv[5], hv[6], hv[7]);
            }
          }
          tc::fence_proxy_async_smem();
        }
        tc::fence_before_sync();
        __syncthreads();  // A[i % 2] written; the epilogue of block i - 2 has read accumulator i % 2
        tc::fence_after_sync();
        if (i < nb && t == 0) {
          const uint32_t acc = tmem + (uint32_t)((i & 1) * kSTN);
          const uint32_t a = tc::smem_u32(sA + (i & 1) * P::kBytesA);
          const uint32_t bh = tc::smem_u32(sBh), bl = tc::smem_u32(sBl);
          for (int ks = 0; ks < nks; ++ks) {
            tc::mma<true>(acc, tc::desc_sw128(a + ks * 32), tc::desc_sw128(bh + ks * 32), idesc, ks != 0);
            tc::mma<true>(acc, tc::desc_sw128(a + ks * 32), tc::desc_sw128(bl + ks * 32), idesc, 1u);
          }
          tc::mma_commit(&mbar[i & 1]);
          issued = true;
        }
        if (i >= 1) {
          // ---- epilogue of block i - 1
          const uint32_t e = (i - 1) & 1;
          const bool ok_wait = tc::mbar_wait(&mbar[e], (ph >> e) & 1u);
          ph ^= 1u << e;
          if (__syncthreads_or(!ok_wait)) {
            failed = true;
            break;
          }
          tc::fence_after_sync();
          const size_t b = b0 + i - 1;
          const bool valid = (uint32_t)(b - gb0) * kBlockRows + t < n_g;
          const float cv = c_prev * (1.f - 1.f / 16384.f);
          const uint8_t* arow = sA + e * P::kBytesA;
          bool have_z = false;
          float z[RT];
          float rho_i = 0.f;
          for (int c0 = 0; c0 < N; c0 += 32) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + e * kSTN + c0, v);
            uint32_t cmask = 0;  // columns where this row is a candidate
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              const int j = c0 + jj;
              const float4 pc = spc[j];
              const bool cand =
                  j < np && valid && (pc.w + rmin_prev <= pc.z) && ((pc.x + cv) - pc.y * v[jj] <= pc.z);
              cmask |= (uint32_t)cand << jj;
            }
            uint32_t wmask = __reduce_or_sync(0xffffffffu, cmask);
            while (wmask) {  // warp-uniform walk over the columns with a candidate
              const int jj = __ffs(wmask) - 1;
              wmask &= wmask - 1u;
              const int j = c0 + jj;
              const float4 pc = spc[j];
              bool ok = false;
              float D = 0.f;
              if ((cmask >> jj) & 1u) {
                if (!have_z) {
#pragma unroll
                  for (int k = 0; k < RT; ++k)
                    z[k] = k < rp ? __half2float(*reinterpret_cast<const __half*>(arow + sw128_off(t, 2 * k))) * s_g
                                  : 0.f;
                  rho_i = rho[b * kBlockRows + t];
                  have_z = true;
                }
                D = eval_D<RT>(sz + j * RT, z, pc.w, rho_i);
                ok = D <= pc.z;
                if (ok && filter) {
                  const long long av = (long long)attr_b[b * kBlockRows + t];
                  ok = av >= slo[j] && av <= shi[j];
                }
              }
              const unsigned mask = __ballot_sync(0xffffffffu, ok);
              if (mask) {
                const int leader = __ffs(mask) - 1;
                uint32_t base = 0;
                if (lane == leader) base = atomicAdd(&cnt[sqid[j]], (uint32_t)__popc(mask));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (ok) {
                  const uint32_t pos = base + __popc(mask & lt_mask);
                  if (pos < cap)
                    surv[(size_t)sqid[j] * cap + pos] =
                        ((unsigned long long)__float_as_uint(D) << 32) | ids[b * kBlockRows + t];
                }
              }
            }
          }
          tc::fence_before_sync();
        }
        c_prev = c_cur;
        rmin_prev = rmin_cur;
#pragma unroll
        for (int l = 0; l < kL; ++l) cur[l] = nxt[l];
        c_cur = c_nxt;
        rmin_cur = rmin_nxt;
        if (i + 2 < nb) load_block(i + 2, nxt, c_nxt, rmin_nxt);
      }
    }
  }
  if (t == 0 && issued) {  // every MMA has completed before TMEM is released
    tc::mma_commit(&fin);
    if (!tc::mbar_wait(&fin, 0)) failed = true;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 2 * kSTN);
  }
  if (t == 0 && failed) atomicOr(err, tc::kErrTimeout);
}

}  // namespace
}  // namespace hntl
