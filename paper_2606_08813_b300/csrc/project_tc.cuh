// Query projection on the tensor cores for the precision form (Eq. 1-4 with
// BF16 query, centres and bases).
//
// Two A operands per K step: the pairs' BF16 query rows q_b and, on the same
// rows, the negated centre -mu_b of each pair's grain; the B operand holds
// the grains' BF16 bases U_g (r rows each, K-major).
// Per K step of 16 the MMA pair adds U_g q_b - U_g mu_b over those 16
// coordinates to the TMEM accumulator, so the accumulator always holds the
// partial z = U_g (q_b - mu_b) of the coordinates seen so far: BF16 products
// are exact and the FP32 accumulation never carries the large |U_g q_b|, which
// keeps the accuracy of the direct form. The residual norm uses the identity,
// valid for any U when z = U v',
//   ||v' - U^T z||^2 = ||v'||^2 - 2 ||z||^2 + z^T (U U^T) z,
// with ||v'||^2 = ||q_b - mu_b||^2 taken from routing (the exact direct-form
// distance of this very pair) and the grain's Gram matrix precomputed.
#pragma once

#include <cuda_bf16.h>

#include "hntl_internal.cuh"
#include "tc_common.cuh"

namespace hntl {
namespace {

constexpr int kPTM = 128;                 // MMA M: 4 slots of 32 pair rows (one TMEM lane quarter each)
constexpr int kPSlot = 32;                // pairs per slot
constexpr int kPSlots = kPTM / kPSlot;    // slots per work item
constexpr int kPKB = 64;                  // BF16 elements per K block (128 bytes)
constexpr uint32_t kPBytesA = kPTM * 128; // one A operand per K block
constexpr int kPThreads = 288;            // 4 producer warps, 1 MMA warp, 4 epilogue warps

template <int RN>
struct ProjTc {
  static constexpr int kN = kPSlots * RN;                              // MMA N: the 4 slots' bases
  static constexpr uint32_t kBytesB = kN * 128;
  static constexpr uint32_t kStage = 2 * kPBytesA + kBytesB;
  static constexpr int kStages = RN <= 16 ? 5 : (RN <= 32 ? 4 : 2);  // ring of K blocks
  static constexpr int kTmemCols = 2 * kN;                            // two accumulators
  static constexpr int kGramRegs = RN <= 32 ? RN * RN / 32 : 0;       // staged per lane (else loaded directly)
  static constexpr int kSmem = kStages * kStage + kPSlots * RN * RN * 4 + 1024;
  static_assert(kTmemCols >= 32 && kTmemCols <= 512 && (kTmemCols & (kTmemCols - 1)) == 0, "TMEM columns");
};

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_val(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// swizzled byte offset of (row, byte) in a K-major 128B-swizzled tile
__device__ __forceinline__ uint32_t sw128_off(int row, int byte) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((byte >> 4) ^ (row & 7)) << 4) | (byte & 15)));
}

// Persistent, warp-specialised projection. The bucket stage cuts each grain's
// pair list into slots of at most 32 pairs; a work item is 4 consecutive
// slots (possibly of 4 different grains). Slot j owns A rows 32j..32j+31 and
// B rows j*RN..j*RN+RN-1 (its grain's basis, zero past r), so TMEM lane
// quarter j, columns j*RN.., holds z of slot j's pairs; the other columns
// (pairs against the other slots' bases) are computed and ignored.
// CTA b takes items b, b + grid, ...
//   warps 0-3  producers: per K block of 64 coordinates, 16-byte asynchronous
//              copies (cp.async, through L2) of the pairs' query chunks and,
//              on the same rows, of the negated centre of each slot's grain
//              (a negated BF16 copy of the centres), straight into the
//              stage's swizzled A tiles, with up to kPDepth K blocks in
//              flight per thread; a thread announces a stage on `full` once
//              its copies into it have landed (wait_group, then the proxy
//              fence that shows them to the tensor cores). TMA brings the 4
//              bases (one load each) into the same stage, counted on `full`
//              by transaction bytes.
//   warp 4     one thread issues the MMAs (+U q_b then -U mu_b per 16
//              coordinates) into one of two TMEM accumulators, frees each
//              stage through `empty` and hands the item on through `accf`.
//   warps 5-8  epilogue, warp w for slot w % 4: read its z, free the
//              accumulator through `acce`, store; with kRho also rho from
//              the Gram identity (the next item's Gram matrix and ||v'||^2
//              are loaded meanwhile), else the explicit-residual pass
//              (k_resid_tc) computes rho.
// RN = basis rows padded to a multiple of 16, r <= RN; d % 8 == 0 (16-byte TMA row strides).
template <int RN, bool kRho>
__global__ void __launch_bounds__(kPThreads, 1) k_project_tc(
    const uint16_t* __restrict__ Qh, const uint16_t* __restrict__ Mhn,
    const __grid_constant__ CUtensorMap mapU, const float* __restrict__ gram, int d, int r,
    const uint4* __restrict__ slots,
    const uint32_t* __restrict__ n_slots, const uint32_t* __restrict__ pair_q, const float* __restrict__ pair_vn,
    float* __restrict__ zq, float* __restrict__ rhoq, int* __restrict__ err) {
  using P = ProjTc<RN>;
  constexpr int S = P::kStages;
  constexpr int kPDepth = S < 3 ? S : 3;  // K blocks of copies in flight per producer thread (<= S)
  constexpr uint32_t kIdesc = tc::idesc_f32acc(1u, kPTM, P::kN);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float* sgram_all = reinterpret_cast<float*>(smem + S * P::kStage);  // [slot][RN][RN]
  __shared__ __align__(8) uint64_t full[S], empty[S], accf[2], acce[2], fin;
  __shared__ uint32_t sq[kPTM];
  __shared__ uint4 sslot[kPSlots];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  __shared__ uint32_t s_it_prod, s_it_mma;  // K blocks issued by the producers / consumed by the MMA thread
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 4) tc::tmem_alloc(&tmem_base, P::kTmemCols);
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], 128);  // every producer arrives once its query row is in
      tc::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(&accf[a], 1);
      tc::mbar_init(&acce[a], 4);
    }
    tc::mbar_init(&fin, 1);
    s_fail = 0;
    s_it_prod = s_it_mma = 0;
    tc::mbar_fence_init();
  }
  if (tid < 128 && r < RN) {  // basis rows r..RN-1 of every slot and stage stay zero
    const int per = kPSlots * (RN - r) * 8;
    for (int e = tid; e < S * per; e += 128) {
      const int s = e / per, rem = e % per, j = rem / ((RN - r) * 8), rr = rem % ((RN - r) * 8);
      const int row = j * RN + r + rr / 8, ch = rr % 8;
      *reinterpret_cast<uint4*>(smem + s * P::kStage + 2 * kPBytesA + sw128_off(row, ch * 16)) =
          make_uint4(0, 0, 0, 0);
    }
    tc::fence_proxy_async_smem();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t ns = *n_slots;
  const uint32_t total = (ns + kPSlots - 1) / kPSlots;
  const int nkb = (d + kPKB - 1) / kPKB;
  auto slot_of = [&](uint32_t w, int j) -> uint4 {
    const uint32_t s = w * kPSlots + j;
    return s < ns ? slots[s] : make_uint4(0, 0, 0, 0);
  };

  if (warp < 4) {
    // ------------------------------------------------------------ producers
    // A row i is pair i % 32 of slot i / 32. Thread t copies 16-byte chunk
    // t % 8 of rows t / 8 + 16 i, i < 8 (so every warp's copies cover 4 whole
    // 128-byte lines), and the same chunk of the negated centre of each of
    // those rows' slots; the bases move by TMA into 1024-byte aligned boxes.
    uint32_t it = 0;   // K blocks issued by this CTA so far
    uint32_t ann = 0;  // K blocks this thread has announced on `full`
    bool failed = false;  // this thread gave up waiting (the MMA thread then gives up too)
    const int my_j = tid >> 5, my_i = tid & 31;
    uint4 nslot = make_uint4(0, 0, 0, 0);
    uint32_t q_next = 0;
    auto prefetch = [&](uint32_t w) {
      const uint4 sl = slot_of(w, my_j);
      q_next = (uint32_t)my_i < sl.z ? pair_q[sl.y + my_i] : 0u;
      if (my_i == 0) nslot = sl;
    };
    // announce the oldest unannounced K block once its copies have landed
    auto announce = [&]() {
      tc::fence_proxy_async_smem();
      tc::mbar_arrive(&full[ann % S]);
      ++ann;
    };
    if (blockIdx.x < total) prefetch(blockIdx.x);
    for (uint32_t w = blockIdx.x; w < total; w += gridDim.x) {
      tc::named_bar(1, 128);  // every producer is done with the previous item's ids
      sq[tid] = q_next;
      if (my_i == 0) sslot[my_j] = nslot;
      if (w + gridDim.x < total) prefetch(w + gridDim.x);
      tc::named_bar(1, 128);
      if (failed) continue;
      const int ch = tid & 7, rbase = tid >> 3;
      uint32_t qok = 0;  // bit i: row rbase + 16 i holds a pair
      const uint16_t* qsrc[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int row = rbase + 16 * i;
        qok |= (uint32_t)((uint32_t)(row & 31) < sslot[row >> 5].z) << i;
        qsrc[i] = Qh + (size_t)sq[row] * d + ch * 8;
      }
      const uint16_t* msrc[kPSlots];
#pragma unroll
      for (int j = 0; j < kPSlots; ++j) msrc[j] = Mhn + (size_t)sslot[j].x * d + ch * 8;
      // TMA bytes one stage receives: the bases of the slots with pairs
      uint32_t bytes = 0;
#pragma unroll
      for (int j = 0; j < kPSlots; ++j) bytes += sslot[j].z ? (uint32_t)r * 128u : 0u;
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int s = (int)(it % S);
        // the MMAs that read this stage S K blocks ago must be done (every
        // producer waits for itself: no barrier between the producer warps)
        if (it >= (uint32_t)S && !tc::mbar_wait(&empty[s], ((it / S) - 1) & 1)) {
          failed = true;
          break;
        }
        uint8_t* st = smem + s * P::kStage;
        const int x = kb * kPKB;
        if (tid == 0) tc::mbar_add_tx(&full[s], bytes);  // before this thread announces the stage
        if (tid < kPSlots && sslot[tid].z)
          tc::tma_load_2d(&mapU, &full[s], st + 2 * kPBytesA + tid * RN * 128, x, (int)sslot[tid].x * r);
        const uint32_t sbase = tc::smem_u32(st);
        const bool in = x + ch * 8 < d;  // d % 8 == 0: a chunk is wholly inside or outside
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if ((qok >> i) & 1u) {
            const uint32_t off = sbase + sw128_off(rbase + 16 * i, ch * 16);
            tc::cp_async16_cg_zfill(off, qsrc[i] + (in ? x : 0), in);  // past d: zeros, nothing read
            // the slot's 32 rows read the same centre chunk: through L1
            tc::cp_async16_ca_zfill(off + kPBytesA, msrc[i >> 1] + (in ? x : 0), in);
          }
        }
        tc::cp_async_commit();
        if (it + 1 - ann >= (uint32_t)kPDepth) {  // keep at most kPDepth - 1 blocks in flight
          tc::cp_async_wait<kPDepth - 1>();
          announce();
        }
      }
    }
    // the last blocks: wait for every copy, then announce what is left
    tc::cp_async_wait<0>();
    while (ann < it) announce();
    atomicMax(&s_it_prod, it);  // a thread that gave up stopped issuing early
    if (failed) atomicExch(&s_fail, 1);
  } else if (warp == 4) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      bool ok = true;
      uint32_t it = 0, li = 0;
      for (uint32_t w = blockIdx.x; w < total && ok; w += gridDim.x, ++li) {
        const int a = (int)(li & 1);
        if (li >= 2 && !tc::mbar_wait(&acce[a], ((li >> 1) - 1) & 1)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t acc = tmem + (uint32_t)(a * P::kN);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % S);
          if (!tc::mbar_wait(&full[s], (it / S) & 1)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_u32(smem + s * P::kStage);
#pragma unroll
          for (int ks = 0; ks < kPKB / 16; ++ks)
#pragma unroll
            for (int part = 0; part < 2; ++part)  // + U q_b, then - U mu_b, over the same 16 coordinates
              tc::mma<true>(acc, tc::desc_sw128(sa + part * kPBytesA + ks * 32),
                            tc::desc_sw128(sa + 2 * kPBytesA + ks * 32), kIdesc, (kb | ks | part) != 0);
          tc::mma_commit(&empty[s]);
        }
        if (ok) tc::mma_commit(&accf[a]);
      }
      if (!ok) atomicExch(&s_fail, 1);
      s_it_mma = it;  // stages whose loads were waited for
      if (it > 0) {
        tc::mma_commit(&fin);  // arrives once every MMA issued above has completed
        if (!tc::mbar_wait(&fin, 0)) atomicExch(&s_fail, 1);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int j = warp & 3;  // slot = TMEM lane quarter of this warp
    float* sgram = sgram_all + j * RN * RN;
    bool failed = false;
    constexpr int kG = kRho ? P::kGramRegs : 0;
    float gnext[kG > 0 ? kG : 1];
    float vn_next = 0.f;
    uint4 sl_next = make_uint4(0, 0, 0, 0);
    auto prefetch = [&](uint32_t w) {
      sl_next = slot_of(w, j);
      if constexpr (kG > 0) {
#pragma unroll
        for (int t = 0; t < kG; ++t) {
          const int e = lane + 32 * t, ga = e / RN, gb = e % RN;
          gnext[t] = (sl_next.z && ga < r && gb < r) ? gram[((size_t)sl_next.x * r + ga) * r + gb] : 0.f;
        }
      }
      if constexpr (kRho) vn_next = (uint32_t)lane < sl_next.z ? pair_vn[sl_next.y + lane] : 0.f;
    };
    if (blockIdx.x < total) prefetch(blockIdx.x);
    uint32_t li = 0;
    for (uint32_t w = blockIdx.x; w < total; w += gridDim.x, ++li) {
      const uint4 sl = sl_next;
      const float vn = vn_next;
      __syncwarp();  // this warp is done reading its previous Gram matrix
      if constexpr (!kRho) {
      } else if constexpr (kG > 0) {
#pragma unroll
        for (int t = 0; t < kG; ++t) sgram[lane + 32 * t] = gnext[t];
      } else {
        for (int e = lane; e < RN * RN; e += 32) {
          const int ga = e / RN, gb = e % RN;
          sgram[e] = (sl.z && ga < r && gb < r) ? gram[((size_t)sl.x * r + ga) * r + gb] : 0.f;
        }
      }
      __syncwarp();
      if (w + gridDim.x < total) prefetch(w + gridDim.x);
      if (failed) continue;
      const int a = (int)(li & 1);
      if (__any_sync(0xffffffffu, !tc::mbar_wait(&accf[a], (li >> 1) & 1))) {  // warp-uniform
        failed = true;
        continue;
      }
      tc::fence_after_sync();
      const int np = (int)sl.z;
      float z[RN];
      if (np > 0) {
        const uint32_t taddr = tmem + ((uint32_t)(j * 32) << 16) + (uint32_t)(a * P::kN + j * RN);
        if constexpr (RN == 16) {
          float v[16];
          tc::tmem_ld16(taddr, v);
#pragma unroll
          for (int c = 0; c < 16; ++c) z[c] = v[c];
        } else {
#pragma unroll
          for (int c0 = 0; c0 < RN; c0 += 32) {
            float v[32];
            tc::tmem_ld32(taddr + c0, v);
#pragma unroll
            for (int c = 0; c < 32; ++c) z[c0 + c] = v[c];
          }
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acce[a]);
      if (lane < np) {
        const uint32_t pr = sl.y + lane;
        if constexpr (kRho) {
          float zz = 0.f, qf = 0.f;
#pragma unroll
          for (int ia = 0; ia < RN; ++ia) {
            zz = fmaf(z[ia], z[ia], zz);
            float acc = 0.f;
#pragma unroll
            for (int ib = 0; ib < RN; ++ib) acc = fmaf(sgram[ia * RN + ib], z[ib], acc);
            qf = fmaf(z[ia], acc, qf);
          }
          const float rho = (vn - 2.f * zz) + qf;
          rhoq[pr] = rho > 0.f ? rho : 0.f;
        }
        float* out = zq + (size_t)pr * r;
        if ((r & 3) == 0) {
#pragma unroll
          for (int ia = 0; ia < RN; ia += 4)
            if (ia < r) *reinterpret_cast<float4*>(out + ia) = make_float4(z[ia], z[ia + 1], z[ia + 2], z[ia + 3]);
        } else {
#pragma unroll
          for (int ia = 0; ia < RN; ++ia)
            if (ia < r) out[ia] = z[ia];
        }
      }
    }
    if (failed) atomicExch(&s_fail, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0 && s_fail) {
    // loads issued but never waited for (a wait gave up): let them land before the CTA exits
    for (uint32_t j = s_it_mma; j < s_it_prod; ++j) tc::mbar_wait(&full[j % S], (j / S) & 1, 1u << 16);
  }
  if (warp == 4) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, P::kTmemCols);
  }
  if (tid == 0 && s_fail) atomicOr(err, tc::kErrTimeout);
}

// The distinct grains of an item's slots: the slots with pairs come first and
// a grain's slots are consecutive, so each new grain follows the last one
// seen. nd of them, slot j's distinct index in u_of[j] (0 for a slot without
// pairs), the grain of distinct index u from grain(). The residual passes
// give each distinct grain, not each slot, a K range of their block-diagonal
// A and load each distinct basis once, so the K steps of an item whose slots
// share grains are fewer. (The projections keep one MMA over all 4 slots'
// bases: one N = 4 RN product measured faster than an N = RN product per
// distinct grain.)
struct ItemGrains {
  int nd;
  int u_of[kPSlots];
  // the grain of distinct index u (u < nd)
  __device__ __forceinline__ uint32_t grain(const uint4* sl, int u) const {
    uint32_t g = 0;
#pragma unroll
    for (int j = kPSlots - 1; j >= 0; --j)
      if (sl[j].z && u_of[j] == u) g = sl[j].x;
    return g;
  }
};
__device__ __forceinline__ ItemGrains item_grains(const uint4* sl) {
  ItemGrains ig;
  ig.nd = sl[0].z ? 1 : 0;
  ig.u_of[0] = 0;
#pragma unroll
  for (int j = 1; j < kPSlots; ++j) {
    const bool fresh = sl[j].z && sl[j].x != sl[j - 1].x;
    ig.u_of[j] = sl[j].z ? ig.u_of[j - 1] + (fresh ? 1 : 0) : 0;
    ig.nd += fresh ? 1 : 0;
  }
  return ig;
}

// ------------------------------------------------------------------ explicit residual

// rho_q = ||v' - U_b^T z||^2 of every pair (Eq. 3-4 in the precision form,
// v' = q_b - mu_b), from the z the projection wrote. The Gram identity above
// is exact for the exact z but amplifies the FP32 error dz of the computed z
// into rho by -2 z . dz, which for a query near a grain's subspace but far
// from its centre (|z|^2 >> rho) exceeds 1e-5 of the distance; the explicit
// residual moves only by 2 (z - G z) . dz + |U^T dz|^2 (G = U_b U_b^T is the
// identity to BF16 precision), so this pass recomputes it.
// Work items are the projection's: 4 slots of up to 32 pairs. The
// reconstruction U_b^T z of all 128 pairs against a 128-coordinate chunk is
// one MMA sequence: A = z split into two BF16 parts (hi, lo: 16 significant
// bits; the dropped remainder eta moves rho by 2 (U e) . eta + |U^T eta|^2,
// with U e = (I - G) z + dz small), block-diagonal over the item's distinct
// grains (row i holds its z in K columns u RN .. u RN + RN - 1, u its slot's
// distinct grain, zeros elsewhere; only the K steps of those grains run);
// B = those grains' basis rows for the 128 coordinates, TMA boxes of 64
// coordinates x r rows read MN-major (K = basis row, N = coordinate). TMEM
// lane i, column t then holds (U^T z)_t of pair i; the epilogue adds
// (q_b - mu_b - that)^2.
//   warp 0     TMA producer: per chunk, 2 boxes per distinct grain into a stage ring.
//   warp 1     one thread issues the MMAs into one of two TMEM accumulators.
//   warps 2-9  epilogue: warp w reads lane quarter w % 4 (32 pairs), columns
//              64 (w - 2) / 4 .. + 63 of each chunk; it also writes the A
//              operand of each item before the item's MMAs.
constexpr int kRThr = 320;
constexpr int kRStg = 3;
constexpr int kRChunk = 128;  // coordinates per MMA (N)

constexpr int kRMuD = 1024;  // centre rows of an item are staged in shared memory up to this d
constexpr int kRParts = 2;   // BF16 parts of z (hi, lo: 16 significant bits)

template <int RN>
struct ResidTc {
  static constexpr int kK = kPSlots * RN;                       // A's K: the 4 slots' basis rows
  static constexpr uint32_t kBytesApart = kPTM * kK * 2;         // one part of A (128 rows x kK BF16)
  static constexpr uint32_t kBytesSlot = 2 * RN * 128;           // one slot's 2 boxes of a chunk
  static constexpr uint32_t kStage = kPSlots * kBytesSlot;
  static constexpr uint32_t kBytesMu = kPSlots * kRMuD * 2;     // the item's 4 BF16 centre rows
  static constexpr uint32_t kQRow = 144;                         // a pair's 64 query values, padded
  static constexpr uint32_t kBytesQ = 8 * 32 * kQRow;            // per epilogue warp, its 32 rows
  static constexpr int kSmem = kRParts * kBytesApart + kRStg * kStage + kBytesMu + kBytesQ + 1024;
  static_assert(kSmem <= 227 * 1024, "shared memory per CTA");
};

__device__ __forceinline__ uint16_t bf16_rn(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }

template <int RN>
__global__ void __launch_bounds__(kRThr, 1) k_resid_tc(
    const uint16_t* __restrict__ Qh, const uint16_t* __restrict__ Mh, const __grid_constant__ CUtensorMap mapU,
    int d, int r, const uint4* __restrict__ slots, const uint32_t* __restrict__ n_slots,
    const uint32_t* __restrict__ pair_q, const float* __restrict__ zq, float* __restrict__ rhoq,
    int* __restrict__ err) {
  using P = ResidTc<RN>;
  static_assert(P::kK % 64 == 0 || P::kK == 64, "A rows are whole 128-byte swizzle atoms");
  constexpr int kAtomsK = P::kK / 64;  // 128-byte K atoms per A row
  constexpr uint32_t kIdesc = tc::idesc_f32acc_bmn(1u, kPTM, kRChunk);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;                            // [kRParts][kAtomsK][128 rows x 128 B]
  uint8_t* sB = smem + kRParts * P::kBytesApart; // [stage][slot][2 boxes][RN rows x 128 B]
  uint16_t* sMu = reinterpret_cast<uint16_t*>(sB + kRStg * P::kStage);  // [slot][d] when d <= kRMuD
  uint8_t* sQall = reinterpret_cast<uint8_t*>(sMu) + P::kBytesMu;        // [epilogue warp][32 rows][kQRow]
  __shared__ __align__(8) uint64_t full[kRStg], empty[kRStg], accf[2], acce[2], afull, fin;
  __shared__ uint4 sslot[kPSlots];
  __shared__ float sred[kPTM];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  __shared__ uint32_t s_it_prod, s_it_mma;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 1) tc::tmem_alloc(&tmem_base, 2 * kRChunk);
  if (tid == 0) {
    for (int s = 0; s < kRStg; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(&accf[a], 1);
      tc::mbar_init(&acce[a], 8);
    }
    tc::mbar_init(&afull, 1);
    tc::mbar_init(&fin, 1);
    s_fail = 0;
    s_it_prod = s_it_mma = 0;
    tc::mbar_fence_init();
  }
  // The whole basis ring starts at zero: rows r .. RN - 1 of every box stay
  // zero (TMA writes r rows), and a slot without pairs multiplies its (stale
  // or never written) tile by the zeros of A, which must therefore be finite.
  // A starts at zero too: outside each row's own slot range it stays zero for
  // good, and inside it a row without a pair keeps finite stale values whose
  // output nobody reads.
  for (uint32_t e = tid; e < (uint32_t)(kRStg * P::kStage / 16); e += kRThr)
    *reinterpret_cast<uint4*>(sB + (size_t)e * 16) = make_uint4(0, 0, 0, 0);
  for (uint32_t e = tid; e < (uint32_t)(kRParts * P::kBytesApart / 16); e += kRThr)
    *reinterpret_cast<uint4*>(sA + (size_t)e * 16) = make_uint4(0, 0, 0, 0);
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t ns = *n_slots;
  const uint32_t total = (ns + kPSlots - 1) / kPSlots;
  const int nch = (d + kRChunk - 1) / kRChunk;
  auto slot_of = [&](uint32_t w, int j) -> uint4 {
    const uint32_t s = w * kPSlots + j;
    return s < ns ? slots[s] : make_uint4(0, 0, 0, 0);
  };

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (uint32_t w = blockIdx.x; w < total && ok; w += gridDim.x) {
        uint4 sl[kPSlots];
#pragma unroll
        for (int j = 0; j < kPSlots; ++j) sl[j] = slot_of(w, j);
        const ItemGrains ig = item_grains(sl);
        const uint32_t bytes = (uint32_t)ig.nd * 2u * (uint32_t)r * 128u;
        for (int c = 0; c < nch; ++c, ++it) {
          const int s = (int)(it % kRStg);
          if (it >= (uint32_t)kRStg && !tc::mbar_wait(&empty[s], ((it / kRStg) - 1) & 1)) {
            ok = false;
            break;
          }
          uint8_t* st = sB + s * P::kStage;
          tc::mbar_expect_tx(&full[s], bytes);
#pragma unroll
          for (int u = 0; u < kPSlots; ++u)
            if (u < ig.nd) {
              const int gy = (int)ig.grain(sl, u) * r;
              tc::tma_load_2d(&mapU, &full[s], st + u * P::kBytesSlot, c * kRChunk, gy);
              tc::tma_load_2d(&mapU, &full[s], st + u * P::kBytesSlot + RN * 128, c * kRChunk + 64, gy);
            }
        }
      }
      s_it_prod = it;
      if (!ok) atomicExch(&s_fail, 1);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      bool ok = true;
      uint32_t it = 0, li = 0, ci = 0;  // stage uses, items, accumulator uses
      // every MMA's operand descriptors, once: A per (part, K step); B per K step
      // for stage 0 (another stage adds its byte offset / 16 to the start field)
      constexpr int kKS = P::kK / 16;
      uint64_t da[kRParts][kKS], db0[kKS];
#pragma unroll
      for (int part = 0; part < kRParts; ++part)
#pragma unroll
        for (int ks = 0; ks < kKS; ++ks)
          da[part][ks] = tc::desc_sw128(tc::smem_u32(sA + part * P::kBytesApart) + (ks / 4) * (kPTM * 128) +
                                        (ks % 4) * 32);
#pragma unroll
      for (int ks = 0; ks < kKS; ++ks)
        db0[ks] = tc::desc_sw128_mn(tc::smem_u32(sB) + (ks / (RN / 16)) * P::kBytesSlot + (ks % (RN / 16)) * 2048,
                                    RN * 128);
      for (uint32_t w = blockIdx.x; w < total && ok; w += gridDim.x, ++li) {
        if (!tc::mbar_wait(&afull, li & 1)) {  // this item's A operand is written
          ok = false;
          break;
        }
        tc::fence_after_sync();
        uint4 slw[kPSlots];
#pragma unroll
        for (int j = 0; j < kPSlots; ++j) slw[j] = slot_of(w, j);
        const int nks = item_grains(slw).nd * (RN / 16);  // K steps of the distinct grains' ranges
        for (int c = 0; c < nch; ++c, ++it, ++ci) {
          const int s = (int)(it % kRStg), a = (int)(ci & 1);
          if (ci >= 2 && !tc::mbar_wait(&acce[a], ((ci >> 1) - 1) & 1)) {
            ok = false;
            break;
          }
          if (!tc::mbar_wait(&full[s], (it / kRStg) & 1)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t acc = tmem + (uint32_t)(a * kRChunk);
          const uint64_t soff = (uint64_t)((s * P::kStage) >> 4);  // stays inside the 14-bit start field
#pragma unroll
          for (int part = 0; part < kRParts; ++part)
#pragma unroll
            for (int ks = 0; ks < kKS; ++ks)
              if (ks < nks) tc::mma<true>(acc, da[part][ks], db0[ks] + soff, kIdesc, (part | ks) != 0);
          tc::mma_commit(&empty[s]);
          tc::mma_commit(&accf[a]);
        }
      }
      if (!ok) atomicExch(&s_fail, 1);
      s_it_mma = it;
      if (it > 0) {
        tc::mma_commit(&fin);
        if (!tc::mbar_wait(&fin, 0)) atomicExch(&s_fail, 1);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ A operand and epilogue
    const int et = tid - 64;                // 0 .. 255
    const int q4 = warp & 3;                // TMEM lane quarter = slot
    const int half = (warp - 2) >> 2;       // 0: columns 0..63 of a chunk, 1: 64..127
    const int row = q4 * 32 + lane;         // A row = TMEM lane = pair of the item
    bool failed = false;
    uint32_t li = 0, ci = 0;
    // this thread's A row (two threads per row, RN / 2 of its values each) and
    // the next item's slot record and z values, loaded while the current item runs
    const int ra = et >> 1, hf = et & 1, sa = ra / 32, ia = ra % 32;
    constexpr int kH = RN / 2;
    float zn[kH];
    bool zn_have = false;
    auto prefetch_z = [&](uint32_t w) {
      const uint4 sla = slot_of(w, sa);
      zn_have = (uint32_t)ia < sla.z;
      const float* z = zq + (size_t)(sla.y + (zn_have ? ia : 0)) * r;
#pragma unroll
      for (int j = 0; j < kH; ++j) {
        const int jj = hf * kH + j;
        zn[j] = (zn_have && jj < r) ? z[jj] : 0.f;
      }
    };
    if (blockIdx.x < total) prefetch_z(blockIdx.x);
    int prev_u = -1;  // the K range this thread's pieces of its row were last written to
    for (uint32_t w = blockIdx.x; w < total; w += gridDim.x, ++li) {
      if (et < kPSlots) sslot[et] = slot_of(w, et);
      // A: row i holds its z at K = u RN .. u RN + RN - 1, u the distinct grain
      // of its slot (kRParts BF16 parts: hi = bf16(v), lo = bf16(v - hi);
      // v - hi - lo is below 2^-16 |v|); a range a row leaves is zeroed
      {
        int ua = 0;
        if (zn_have) {
          uint4 slw[kPSlots];
#pragma unroll
          for (int j = 0; j < kPSlots; ++j) slw[j] = slot_of(w, j);
          const ItemGrains igw = item_grains(slw);
#pragma unroll
          for (int j = 0; j < kPSlots; ++j)
            if (j == sa) ua = igw.u_of[j];
          if (prev_u >= 0 && prev_u != ua) {
#pragma unroll
            for (int c8 = 0; c8 < kH / 8; ++c8) {
              const int kc = (prev_u * RN + hf * kH) / 8 + c8;
#pragma unroll
              for (int part = 0; part < kRParts; ++part)
                *reinterpret_cast<uint4*>(sA + part * P::kBytesApart + (kc / 8) * (kPTM * 128) +
                                          sw128_off(ra, (kc % 8) * 16)) = make_uint4(0, 0, 0, 0);
            }
          }
          prev_u = ua;
        }
        if (zn_have) {
          float zv[kH];
#pragma unroll
          for (int j = 0; j < kH; ++j) zv[j] = zn[j];
#pragma unroll
          for (int c8 = 0; c8 < kH / 8; ++c8) {  // 16-byte chunks of 8 values
            uint32_t wp[kRParts][4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              uint32_t w2[kRParts] = {};
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                float v = zv[c8 * 8 + 2 * h + u];
#pragma unroll
                for (int part = 0; part < kRParts; ++part) {  // successive BF16 parts of the remainder
                  const uint16_t b = bf16_rn(v);
                  w2[part] |= (uint32_t)b << (16 * u);
                  v -= bf16_val(b);
                }
              }
#pragma unroll
              for (int part = 0; part < kRParts; ++part) wp[part][h] = w2[part];
            }
            const int kc = (ua * RN + hf * kH) / 8 + c8;  // chunk index along K
#pragma unroll
            for (int part = 0; part < kRParts; ++part)
              *reinterpret_cast<uint4*>(sA + part * P::kBytesApart + (kc / 8) * (kPTM * 128) +
                                        sw128_off(ra, (kc % 8) * 16)) =
                  make_uint4(wp[part][0], wp[part][1], wp[part][2], wp[part][3]);
          }
        }
      }
      tc::fence_proxy_async_smem();
      tc::named_bar(1, 256);
      if (et == 0) tc::mbar_arrive(&afull);
      if (w + gridDim.x < total) prefetch_z(w + gridDim.x);
      const uint4 sl = sslot[q4];
      const bool mine = (uint32_t)lane < sl.z;
      // the warp's 32 query rows move by coalesced loads: load i brings 16-byte
      // piece lane % 8 of row 4 i + lane / 8 (four whole 128-byte lines a load),
      // and a pass through this warp's shared buffer hands every lane its own row
      uint8_t* sQ = sQall + (warp - 2) * (32 * P::kQRow);
      uint32_t qrow4[8];  // the rows this lane loads, as query indices (~0u: no pair)
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const uint32_t rw = 4u * i + (lane >> 3);
        qrow4[i] = rw < sl.z ? pair_q[sl.y + rw] : ~0u;
      }
      // the item's centre rows, read by every pair of a slot: staged in shared memory
      const bool mu_smem = d <= kRMuD;
      if (mu_smem) {
        for (int e = et; e < kPSlots * (d / 8); e += 256) {
          const int j = e / (d / 8), c8 = e % (d / 8);
          *reinterpret_cast<uint4*>(sMu + j * kRMuD + c8 * 8) =
              __ldg(reinterpret_cast<const uint4*>(Mh + (size_t)sslot[j].x * d + c8 * 8));
        }
        tc::named_bar(1, 256);
      }
      const uint16_t* mrow = mu_smem ? sMu + q4 * kRMuD : Mh + (size_t)sl.x * d;
      float acc = 0.f;
      // the 64 coordinates of a chunk this warp handles, loaded one chunk ahead
      uint4 qn[8];
      auto load_q = [&](int c) {
        const int t = c * kRChunk + half * 64 + (lane & 7) * 8;
#pragma unroll
        for (int i = 0; i < 8; ++i)
          qn[i] = (qrow4[i] != ~0u && c < nch && t < d)
                      ? __ldg(reinterpret_cast<const uint4*>(Qh + (size_t)qrow4[i] * d + t))
                      : make_uint4(0, 0, 0, 0);
      };
      load_q(0);
      for (int c = 0; c < nch; ++c, ++ci) {
        const int a = (int)(ci & 1);
        uint4 qv8[8];
        __syncwarp();  // every lane has read the previous chunk's rows
#pragma unroll
        for (int i = 0; i < 8; ++i)
          *reinterpret_cast<uint4*>(sQ + (4 * i + (lane >> 3)) * P::kQRow + (lane & 7) * 16) = qn[i];
        __syncwarp();
#pragma unroll
        for (int g8 = 0; g8 < 8; ++g8) qv8[g8] = *reinterpret_cast<const uint4*>(sQ + lane * P::kQRow + g8 * 16);
        load_q(c + 1);
        if (!failed && __any_sync(0xffffffffu, !tc::mbar_wait(&accf[a], (ci >> 1) & 1))) failed = true;
        if (failed) continue;
        tc::fence_after_sync();
        const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(a * kRChunk + half * 64);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {  // 32 columns at a time
          float v[32];
          tc::tmem_ld32(taddr + 32 * hh, v);
          if (hh == 1) {
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acce[a]);
          }
          if (mine) {
#pragma unroll
            for (int g4 = 0; g4 < 4; ++g4) {
              const int g8 = hh * 4 + g4;
              const int t = c * kRChunk + half * 64 + g8 * 8;
              const uint4 mv = t < d ? *reinterpret_cast<const uint4*>(mrow + t) : make_uint4(0, 0, 0, 0);
              const uint32_t qw[4] = {qv8[g8].x, qv8[g8].y, qv8[g8].z, qv8[g8].w};
              const uint32_t mw[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
              for (int h = 0; h < 4; ++h) {  // zeros past d: q = mu = reconstruction = 0
                const float e0 =
                    (bf16_val((uint16_t)(qw[h] & 0xFFFFu)) - bf16_val((uint16_t)(mw[h] & 0xFFFFu))) - v[g4 * 8 + 2 * h];
                const float e1 =
                    (bf16_val((uint16_t)(qw[h] >> 16)) - bf16_val((uint16_t)(mw[h] >> 16))) - v[g4 * 8 + 2 * h + 1];
                acc = fmaf(e0, e0, acc);
                acc = fmaf(e1, e1, acc);
              }
            }
          }
        }
      }
      // the two column halves of each pair
      if (half == 1) sred[row] = acc;
      tc::named_bar(1, 256);
      if (half == 0 && mine && !failed) rhoq[sl.y + lane] = acc + sred[row];
      tc::named_bar(1, 256);
    }
    if (failed) atomicExch(&s_fail, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0 && s_fail) {
    for (uint32_t j = s_it_mma; j < s_it_prod; ++j) tc::mbar_wait(&full[j % kRStg], (j / kRStg) & 1, 1u << 16);
  }
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 2 * kRChunk);
  }
  if (tid == 0 && s_fail) atomicOr(err, tc::kErrTimeout);
}

// Per grain (BF16 form): the Gram matrix U_g U_g^T (r x r, FP32 sums of exact products).
__global__ void k_gram(const uint16_t* __restrict__ Uh, int d, int r, float* __restrict__ gram) {
  const int g = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int e = warp; e < r * r; e += nw) {
    const int a = e / r, b = e % r;
    const uint16_t* ua = Uh + ((size_t)g * r + a) * d;
    const uint16_t* ub = Uh + ((size_t)g * r + b) * d;
    float acc = 0.f;
    for (int t = lane; t < d; t += 32) acc = fmaf(bf16_val(ua[t]), bf16_val(ub[t]), acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) gram[((size_t)g * r + a) * r + b] = acc;
  }
}

}  // namespace
}  // namespace hntl
