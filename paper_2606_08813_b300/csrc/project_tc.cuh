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
//   warps 0-3  producers: per K block of 64 coordinates, the pairs' query
//              rows and, on the same rows, the negated centre of each slot's
//              grain (coalesced 16-byte loads prefetched one K block ahead,
//              sign flip, swizzled stores, proxy fence, arrival on the
//              stage's `full` barrier); TMA brings the 4 bases (one load
//              each) into the same stage, counted on `full` by transaction
//              bytes.
//   warp 4     one thread issues the MMAs (+U q_b then -U mu_b per 16
//              coordinates) into one of two TMEM accumulators, frees each
//              stage through `empty` and hands the item on through `accf`.
//   warps 5-8  epilogue, warp w for slot w % 4: read its z, free the
//              accumulator through `acce`, rho from the Gram identity, store;
//              the next item's Gram matrix and ||v'||^2 are loaded meanwhile.
// RN = basis rows padded to a multiple of 16, r <= RN; d % 8 == 0 (16-byte TMA row strides).
template <int RN>
__global__ void __launch_bounds__(kPThreads, 1) k_project_tc(
    const uint16_t* __restrict__ Qh, const uint16_t* __restrict__ Mh,
    const __grid_constant__ CUtensorMap mapU, const float* __restrict__ gram, int d, int r,
    const uint4* __restrict__ slots,
    const uint32_t* __restrict__ n_slots, const uint32_t* __restrict__ pair_q, const float* __restrict__ pair_vn,
    float* __restrict__ zq, float* __restrict__ rhoq, int* __restrict__ err) {
  using P = ProjTc<RN>;
  constexpr int S = P::kStages;
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
    // A row i is pair i % 32 of slot i / 32. Query rows and centre chunks move
    // by 16-byte loads, 8 lanes per row, prefetched one K block ahead in
    // registers, and swizzled stores; the bases move by TMA into
    // 1024-byte aligned boxes.
    uint32_t it = 0;  // K blocks issued by this CTA so far
    bool failed = false;  // uniform over the producers (decided by barrier reductions)
    const int my_j = tid >> 5, my_i = tid & 31;
    uint4 nslot = make_uint4(0, 0, 0, 0);
    uint32_t q_next = 0;
    auto prefetch = [&](uint32_t w) {
      const uint4 sl = slot_of(w, my_j);
      q_next = (uint32_t)my_i < sl.z ? pair_q[sl.y + my_i] : 0u;
      if (my_i == 0) nslot = sl;
    };
    if (blockIdx.x < total) prefetch(blockIdx.x);
    for (uint32_t w = blockIdx.x; w < total; w += gridDim.x) {
      tc::named_bar(1, 128);  // every producer is done with the previous item's ids
      sq[tid] = q_next;
      if (my_i == 0) sslot[my_j] = nslot;
      if (w + gridDim.x < total) prefetch(w + gridDim.x);
      tc::named_bar(1, 128);
      if (failed) continue;
      // thread t carries chunk t % 8 of rows t / 8 + 16 i, i < 8 (so every warp
      // load covers 4 whole 128-byte lines); row t / 8 + 16 i belongs to slot i / 2,
      // whose centre chunk the thread also loads
      const int ch = tid & 7, rbase = tid >> 3;
      uint32_t qok = 0;  // bit i: row rbase + 16 i holds a pair
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int row = rbase + 16 * i;
        qok |= (uint32_t)((uint32_t)(row & 31) < sslot[row >> 5].z) << i;
      }
      // TMA bytes one stage receives: the bases of the slots with pairs
      uint32_t bytes = 0;
#pragma unroll
      for (int j = 0; j < kPSlots; ++j) bytes += sslot[j].z ? (uint32_t)r * 128u : 0u;
      uint4 qa[8], ma[kPSlots];
      auto load_q = [&](int kb) {
        const int kk = kb * kPKB + ch * 8;
#pragma unroll
        for (int i = 0; i < 8; ++i)
          qa[i] = ((qok >> i) & 1u) && kk < d
                      ? __ldg(reinterpret_cast<const uint4*>(Qh + (size_t)sq[rbase + 16 * i] * d + kk))
                      : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int j = 0; j < kPSlots; ++j)
          ma[j] = ((qok >> (2 * j)) & 3u) && kk < d
                      ? __ldg(reinterpret_cast<const uint4*>(Mh + (size_t)sslot[j].x * d + kk))
                      : make_uint4(0, 0, 0, 0);
      };
      load_q(0);
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int s = (int)(it % S);
        if (it >= (uint32_t)S) {  // the MMAs that read this stage S K blocks ago must be done
          const bool ok = tid != 0 || tc::mbar_wait(&empty[s], ((it / S) - 1) & 1);
          if (tc::named_bar_or(1, 128, !ok)) {
            failed = true;
            break;
          }
        }
        uint8_t* st = smem + s * P::kStage;
        const int x = kb * kPKB;
        if (tid == 0) tc::mbar_add_tx(&full[s], bytes);  // before this thread's arrival below
        if (tid < kPSlots && sslot[tid].z)
          tc::tma_load_2d(&mapU, &full[s], st + 2 * kPBytesA + tid * RN * 128, x, (int)sslot[tid].x * r);
        const uint32_t sbase = tc::smem_u32(st);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if ((qok >> i) & 1u) {
            const uint32_t off = sbase + sw128_off(rbase + 16 * i, ch * 16);
            const uint4 m = ma[i >> 1];  // -mu_b: flip the sign bit of each BF16 (exact)
            asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(off), "r"(qa[i].x), "r"(qa[i].y),
                         "r"(qa[i].z), "r"(qa[i].w)
                         : "memory");
            asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(off + kPBytesA),
                         "r"(m.x ^ 0x80008000u), "r"(m.y ^ 0x80008000u), "r"(m.z ^ 0x80008000u),
                         "r"(m.w ^ 0x80008000u)
                         : "memory");
          }
        }
        tc::fence_proxy_async_smem();
        tc::mbar_arrive(&full[s]);
        if (kb + 1 < nkb) load_q(kb + 1);
      }
    }
    if (tid == 0) {
      s_it_prod = it;
      if (failed) atomicExch(&s_fail, 1);
    }
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
    float gnext[P::kGramRegs > 0 ? P::kGramRegs : 1];
    float vn_next = 0.f;
    uint4 sl_next = make_uint4(0, 0, 0, 0);
    auto prefetch = [&](uint32_t w) {
      sl_next = slot_of(w, j);
      if constexpr (P::kGramRegs > 0) {
#pragma unroll
        for (int t = 0; t < P::kGramRegs; ++t) {
          const int e = lane + 32 * t, ga = e / RN, gb = e % RN;
          gnext[t] = (sl_next.z && ga < r && gb < r) ? gram[((size_t)sl_next.x * r + ga) * r + gb] : 0.f;
        }
      }
      vn_next = (uint32_t)lane < sl_next.z ? pair_vn[sl_next.y + lane] : 0.f;
    };
    if (blockIdx.x < total) prefetch(blockIdx.x);
    uint32_t li = 0;
    for (uint32_t w = blockIdx.x; w < total; w += gridDim.x, ++li) {
      const uint4 sl = sl_next;
      const float vn = vn_next;
      __syncwarp();  // this warp is done reading its previous Gram matrix
      if constexpr (P::kGramRegs > 0) {
#pragma unroll
        for (int t = 0; t < P::kGramRegs; ++t) sgram[lane + 32 * t] = gnext[t];
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
        float zz = 0.f, qf = 0.f;
#pragma unroll
        for (int ia = 0; ia < RN; ++ia) {
          zz = fmaf(z[ia], z[ia], zz);
          float acc = 0.f;
#pragma unroll
          for (int ib = 0; ib < RN; ++ib) acc = fmaf(sgram[ia * RN + ib], z[ib], acc);
          qf = fmaf(z[ia], acc, qf);
        }
        const uint32_t pr = sl.y + lane;
        const float rho = (vn - 2.f * zz) + qf;
        rhoq[pr] = rho > 0.f ? rho : 0.f;
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
