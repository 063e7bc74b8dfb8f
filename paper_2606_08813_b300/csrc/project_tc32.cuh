// Query projection on the tensor cores for the FP32 form (and the 16-bit
// form, which quantises the FP32 projection): Eq. 1-4 with FP32 queries,
// centres and bases, to FP32 accuracy.
//
// Every FP32 operand x is carried as three BF16 parts, x0 = bf16(x),
// x1 = bf16(x - x0), x2 = bf16(x - x0 - x1) (each remainder is exact in
// FP32), so x - x0 - x1 - x2 is at most 2^-24 |x|. A product a b is formed
// from the six part products a_i b_j with i + j <= 2; the three dropped ones
// and the parts' remainders together stay below about 4 x 2^-24 |a| |b|, the
// size of an FP32 rounding. The accumulation is FP32 in TMEM, in two
// accumulators: the leading products a_0 b_0 in one, the five small cross
// products (about 2^-8 of them) in the other, so that every MMA that adds a
// cross product rounds a sum 2^-8 the size of z; the epilogue adds the two.
//   k_project_tc3  z = U_g (q - mu_g): the producers form v' = q - mu_g in
//                  FP32 (as the direct form does) and split it; the bases'
//                  parts come precomputed (Index::U3) by TMA.
//   k_resid_tc3    rho_q = ||v' - U_g^T z||^2, the explicit residual: the
//                  reconstruction U_g^T z from z's and the bases' parts, the
//                  difference with v' in FP32.
// Work items are those of the precision form's projection: 4 slots of up to
// 32 pairs of one grain each (the bucket stage's slot records).
#pragma once

#include "project_tc.cuh"

namespace hntl {
namespace {

constexpr int kP3Parts = 3;
constexpr int kP3Prod = 6;         // part products (i, j) with i + j <= 2
constexpr int kP3ProdThr = 512;    // 16 producer warps (four per scheduler hide the split's dependent chains)
constexpr int kP3Thr = kP3ProdThr + 160;  // then 4 epilogue warps and 1 MMA warp
constexpr int kP3EpiWarp = kP3ProdThr / 32;
constexpr int kP3MmaWarp = kP3EpiWarp + 4;
constexpr int kP3RowsPer = kPTM * 8 / kP3ProdThr;  // A rows each producer thread fills (one 16-byte piece each)
constexpr int kP3MuD = 1024;       // the item's centre rows are staged in shared memory: d <= this
constexpr int kP3MuPer = kPSlots * kP3MuD / 4 / kP3ProdThr;  // 16-byte centre pieces a producer thread copies

__host__ __device__ constexpr int p3_a(int q) { return q == 2 || q == 4 ? 1 : (q == 5 ? 2 : 0); }
__host__ __device__ constexpr int p3_b(int q) { return q == 1 || q == 4 ? 1 : (q == 3 ? 2 : 0); }

// Two FP32 values rounded to nearest-even BF16 in one conversion: `lo` into
// the low half of the word, `hi` into the high half.
__device__ __forceinline__ uint32_t bf16x2_rn(float lo, float hi) {
  uint32_t w;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(hi), "f"(lo));
  return w;
}

// three BF16 parts of 8 FP32 values, packed two to a word (the even value in
// the low half)
__device__ __forceinline__ void split3_pack(const float (&v)[8], uint4 (&out)[kP3Parts]) {
  uint32_t w[kP3Parts][4];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    float a = v[2 * h], b = v[2 * h + 1];
#pragma unroll
    for (int p = 0; p < kP3Parts; ++p) {
      const uint32_t x = bf16x2_rn(a, b);
      w[p][h] = x;
      a -= __uint_as_float(x << 16);  // exact: the remainder of a BF16 rounding
      b -= __uint_as_float(x & 0xFFFF0000u);
    }
  }
#pragma unroll
  for (int p = 0; p < kP3Parts; ++p) out[p] = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
}

template <int RN>
struct ProjTc3 {
  static constexpr int kN = kPSlots * RN;                                // MMA N: the 4 slots' bases
  static constexpr uint32_t kBytesB = kN * 128;                          // one part of B, one K block
  static constexpr uint32_t kStage = kP3Parts * (kPBytesA + kBytesB);    // [A parts][B parts]
  static constexpr int kStages = 2;
  static constexpr uint32_t kBytesMu = 2 * kPSlots * kP3MuD * 4;      // two items' centre rows
  static constexpr int kTmemCols = 4 * kN;                               // two items x (leading, cross)
  static constexpr int kSmem = kStages * kStage + kBytesMu + 1024;
  static_assert(kTmemCols >= 32 && kTmemCols <= 512 && (kTmemCols & (kTmemCols - 1)) == 0, "TMEM columns");
  static_assert(kSmem <= 225 * 1024, "shared memory per CTA");
};

// Persistent and warp-specialised like k_project_tc (slot j of an item owns
// A rows 32j..32j+31, B rows j RN..j RN + RN - 1 and TMEM lane quarter j).
//   warps 0-15 producers: thread t forms, per K block of 64 coordinates, the
//              16-byte pieces t % 8 of A rows t / 8 + 64 i, i < 2 (slots
//              t / 256 and 2 + t / 256): v' = q - mu in FP32 from the query row (registers,
//              loaded one K block ahead) and the slot's centre (staged in
//              shared memory once per item), split into three parts written
//              to the stage's three swizzled A tiles; it then announces the
//              stage on `full`. TMA brings the 4 bases' three parts.
//   warps 16-19 epilogue: z of slot warp % 4 from TMEM to zq.
//   warp 20    one thread issues the six part products per 16 coordinates.
// RN = basis rows padded to 16 or 32, r <= RN; d % 8 == 0, d <= kP3MuD.
template <int RN>
__global__ void __launch_bounds__(kP3Thr, 1) k_project_tc3(
    const float* __restrict__ Q, const float* __restrict__ M, const __grid_constant__ CUtensorMap mapU3, int G,
    int d, int r, const uint4* __restrict__ slots, const uint32_t* __restrict__ n_slots,
    const uint32_t* __restrict__ pair_q, float* __restrict__ zq, int* __restrict__ err) {
  using P = ProjTc3<RN>;
  constexpr int S = P::kStages;
  constexpr uint32_t kIdesc = tc::idesc_f32acc(1u, kPTM, P::kN);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float* sMu = reinterpret_cast<float*>(smem + S * P::kStage);  // [item parity][slot][kP3MuD]
  __shared__ __align__(8) uint64_t full[S], empty[S], accf[2], acce[2], fin;
  __shared__ uint32_t sq[kPTM];
  __shared__ uint4 sslot[kPSlots];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  __shared__ uint32_t s_it_prod, s_it_mma;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == kP3MmaWarp) tc::tmem_alloc(&tmem_base, P::kTmemCols);
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], kP3ProdThr);  // every producer thread arrives once its pieces are written
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
  if (tid < kP3ProdThr && r < RN) {  // basis rows r..RN-1 of every slot, part and stage stay zero
    const int per = kPSlots * (RN - r) * 8;
    for (int e = tid; e < S * kP3Parts * per; e += kP3ProdThr) {
      const int sp = e / per, rem = e % per, j = rem / ((RN - r) * 8), rr = rem % ((RN - r) * 8);
      const int s = sp / kP3Parts, p = sp % kP3Parts;
      const int row = j * RN + r + rr / 8, ch = rr % 8;
      *reinterpret_cast<uint4*>(smem + s * P::kStage + kP3Parts * kPBytesA + p * P::kBytesB +
                                sw128_off(row, ch * 16)) = make_uint4(0, 0, 0, 0);
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

  if (warp < kP3EpiWarp) {
    // ------------------------------------------------------------ producers
    const int pt = tid;
    uint32_t it = 0;       // stages this thread has announced
    bool failed = false;   // this thread gave up waiting (the MMA thread then gives up too)
    const int my_j = pt >> 5, my_i = pt & 31;  // threads < 128: pair my_i of slot my_j
    uint4 nslot = make_uint4(0, 0, 0, 0);
    uint32_t q_next = 0;
    const int d4 = d / 4;
    // the next item's pair ids (registers) and centre rows (asynchronous
    // copies into the other half of sMu, which nobody reads any more)
    auto prefetch = [&](uint32_t w, int buf) {
      if (pt < 128) {
        const uint4 sl = slot_of(w, my_j);
        q_next = (uint32_t)my_i < sl.z ? pair_q[sl.y + my_i] : 0u;
        if (my_i == 0) nslot = sl;
      }
      float* dst = sMu + buf * (kPSlots * kP3MuD);
#pragma unroll
      for (int u = 0; u < kP3MuPer; ++u) {
        const int e = pt + kP3ProdThr * u;
        if (e < kPSlots * d4) {
          const int j = e / d4, c4 = e % d4;
          tc::cp_async16_ca_zfill(tc::smem_u32(dst + j * kP3MuD + 4 * c4),
                                  M + (size_t)slot_of(w, j).x * d + 4 * c4, true);
        }
      }
      tc::cp_async_commit();
    };
    if (blockIdx.x < total) prefetch(blockIdx.x, 0);
    const int ch = pt & 7, rbase = pt >> 3;  // pieces ch of rows rbase + 64 i, i < 2
    uint32_t li = 0;
    for (uint32_t w = blockIdx.x; w < total; w += gridDim.x, ++li) {
      tc::named_bar(1, kP3ProdThr);  // every producer is done with the previous item's ids and centres
      if (pt < 128) {
        sq[pt] = q_next;
        if (my_i == 0) sslot[my_j] = nslot;
      }
      tc::cp_async_wait<0>();  // this thread's copies of this item's centres have landed
      if (w + gridDim.x < total) prefetch(w + gridDim.x, (int)((li + 1) & 1));
      tc::named_bar(1, kP3ProdThr);   // and everyone else's
      if (failed) continue;
      const float* mu_item = sMu + (li & 1) * (kPSlots * kP3MuD);
      uint32_t qok = 0;  // bit i: row rbase + 64 i holds a pair
      const float* qsrc[kP3RowsPer];
#pragma unroll
      for (int i = 0; i < kP3RowsPer; ++i) {
        const int row = rbase + 64 * i;
        qok |= (uint32_t)((uint32_t)(row & 31) < sslot[row >> 5].z) << i;
        qsrc[i] = Q + (size_t)sq[row] * d + ch * 8;
      }
      uint32_t bytes = 0;  // TMA bytes one stage receives: three parts of each slot's basis
#pragma unroll
      for (int j = 0; j < kPSlots; ++j) bytes += sslot[j].z ? (uint32_t)(kP3Parts * r * 128) : 0u;
      float4 qa[kP3RowsPer][2], qb[kP3RowsPer][2];
      auto load = [&](int kb, float4 (&dst)[kP3RowsPer][2]) {
        const int t = kb * kPKB;
        const bool in = t + ch * 8 < d;  // d % 8 == 0: a piece is wholly inside or outside
#pragma unroll
        for (int i = 0; i < kP3RowsPer; ++i) {
          if (((qok >> i) & 1u) && in) {
            dst[i][0] = __ldg(reinterpret_cast<const float4*>(qsrc[i] + t));
            dst[i][1] = __ldg(reinterpret_cast<const float4*>(qsrc[i] + t + 4));
          } else {
            dst[i][0] = dst[i][1] = make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
      };
      auto stage = [&](int kb, const float4 (&src)[kP3RowsPer][2]) -> bool {
        const int s = (int)(it % S);
        // the MMAs that read this stage S blocks ago must be done (each producer waits for itself)
        if (it >= (uint32_t)S && !tc::mbar_wait(&empty[s], ((it / S) - 1) & 1)) return false;
        uint8_t* st = smem + s * P::kStage;
        const int x = kb * kPKB;
        if (pt == 0) tc::mbar_add_tx(&full[s], bytes);  // before this thread announces the stage
        if (pt < kPSlots * kP3Parts) {
          const int j = pt % kPSlots, p = pt / kPSlots;
          if (sslot[j].z)
            tc::tma_load_2d(&mapU3, &full[s], st + kP3Parts * kPBytesA + p * P::kBytesB + j * RN * 128, x,
                            p * G * r + (int)sslot[j].x * r);
        }
        const bool in = x + ch * 8 < d;
        const uint32_t sbase = tc::smem_u32(st);
#pragma unroll
        for (int i = 0; i < kP3RowsPer; ++i) {
          if (!((qok >> i) & 1u)) continue;  // a row without a pair: its output rows are never read
          const int row = rbase + 64 * i;
          float v[8] = {};
          if (in) {
            const float* mu = mu_item + (row >> 5) * kP3MuD + x + ch * 8;
            const float4 m0 = *reinterpret_cast<const float4*>(mu);
            const float4 m1 = *reinterpret_cast<const float4*>(mu + 4);
            v[0] = src[i][0].x - m0.x;
            v[1] = src[i][0].y - m0.y;
            v[2] = src[i][0].z - m0.z;
            v[3] = src[i][0].w - m0.w;
            v[4] = src[i][1].x - m1.x;
            v[5] = src[i][1].y - m1.y;
            v[6] = src[i][1].z - m1.z;
            v[7] = src[i][1].w - m1.w;
          }
          uint4 parts[kP3Parts];
          split3_pack(v, parts);
          const uint32_t off = sw128_off(row, ch * 16);
#pragma unroll
          for (int p = 0; p < kP3Parts; ++p)
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(sbase + p * kPBytesA + off),
                         "r"(parts[p].x), "r"(parts[p].y), "r"(parts[p].z), "r"(parts[p].w)
                         : "memory");
        }
        tc::fence_proxy_async_smem();  // the generic stores become visible to the tensor cores
        tc::mbar_arrive(&full[s]);
        ++it;
        return true;
      };
      load(0, qa);
      for (int kb = 0; kb < nkb; kb += 2) {
        if (kb + 1 < nkb) load(kb + 1, qb);
        if (!stage(kb, qa)) {
          failed = true;
          break;
        }
        if (kb + 1 >= nkb) break;
        if (kb + 2 < nkb) load(kb + 2, qa);
        if (!stage(kb + 1, qb)) {
          failed = true;
          break;
        }
      }
    }
    tc::cp_async_wait<0>();  // no copy outlives the CTA
    atomicMax(&s_it_prod, it);
    if (failed) atomicExch(&s_fail, 1);
  } else if (warp == kP3MmaWarp) {
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
        const uint32_t acc = tmem + (uint32_t)(a * 2 * P::kN);  // leading products; cross at + kN
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % S);
          if (!tc::mbar_wait(&full[s], (it / S) & 1)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_u32(smem + s * P::kStage);
          const uint32_t sb = sa + kP3Parts * kPBytesA;
#pragma unroll
          for (int ks = 0; ks < kPKB / 16; ++ks)
#pragma unroll
            for (int q = 0; q < kP3Prod; ++q)
              tc::mma<true>(q == 0 ? acc : acc + (uint32_t)P::kN, tc::desc_sw128(sa + p3_a(q) * kPBytesA + ks * 32),
                            tc::desc_sw128(sb + p3_b(q) * P::kBytesB + ks * 32), kIdesc, (kb | ks) != 0 || q > 1);
          tc::mma_commit(&empty[s]);
        }
        if (ok) tc::mma_commit(&accf[a]);
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
    // ------------------------------------------------------------ epilogue
    const int j = warp & 3;  // TMEM lane quarter of this warp = its slot
    bool failed = false;
    uint32_t li = 0;
    for (uint32_t w = blockIdx.x; w < total; w += gridDim.x, ++li) {
      const uint4 sl = slot_of(w, j);
      if (failed) continue;
      const int a = (int)(li & 1);
      if (__any_sync(0xffffffffu, !tc::mbar_wait(&accf[a], (li >> 1) & 1))) {  // warp-uniform
        failed = true;
        continue;
      }
      tc::fence_after_sync();
      const int np = (int)sl.z;
      if (np > 0) {  // leading plus cross products, 16 columns at a time, straight to zq
        const uint32_t taddr = tmem + ((uint32_t)(j * 32) << 16) + (uint32_t)(a * 2 * P::kN + j * RN);
        float* out = zq + (size_t)(sl.y + (lane < np ? lane : 0)) * r;
#pragma unroll
        for (int c0 = 0; c0 < RN; c0 += 16) {
          float v[16], x[16];
          tc::tmem_ld16(taddr + c0, v);
          tc::tmem_ld16(taddr + P::kN + c0, x);
          if (lane < np) {
            if ((r & 3) == 0) {
#pragma unroll
              for (int ia = 0; ia < 16; ia += 4)
                if (c0 + ia < r)
                  *reinterpret_cast<float4*>(out + c0 + ia) =
                      make_float4(v[ia] + x[ia], v[ia + 1] + x[ia + 1], v[ia + 2] + x[ia + 2], v[ia + 3] + x[ia + 3]);
            } else {
#pragma unroll
              for (int ia = 0; ia < 16; ++ia)
                if (c0 + ia < r) out[c0 + ia] = v[ia] + x[ia];
            }
          }
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acce[a]);
    }
    if (failed) atomicExch(&s_fail, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0 && s_fail) {
    // loads issued but never waited for (a wait gave up): let them land before the CTA exits
    for (uint32_t q = s_it_mma; q < s_it_prod; ++q) tc::mbar_wait(&full[q % S], (q / S) & 1, 1u << 16);
  }
  if (warp == kP3MmaWarp) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, P::kTmemCols);
  }
  if (tid == 0 && s_fail) atomicOr(err, tc::kErrTimeout);
}

// ------------------------------------------------------------------ explicit residual

constexpr int kR3Thr = 320;
constexpr int kR3Chunk = 64;  // coordinates per MMA (N)

template <int RN>
struct ResidTc3 {
  static constexpr int kK = kPSlots * RN;                          // A's K: the 4 slots' basis rows
  static constexpr uint32_t kBytesApart = kPTM * kK * 2;            // one part of A (128 rows x kK BF16)
  static constexpr uint32_t kBytesBox = RN * 128;                   // one slot's box of a chunk, one part
  static constexpr uint32_t kBytesBpart = kPSlots * kBytesBox;
  static constexpr uint32_t kStage = kP3Parts * kBytesBpart;        // [part][slot]
  static constexpr int kStages = RN <= 16 ? 3 : 2;
  static constexpr int kSmem = kP3Parts * kBytesApart + kStages * kStage + 1024;
  static_assert(kSmem <= 225 * 1024, "shared memory per CTA");
};

// rho_q = ||v' - U_g^T z||^2 of every pair in FP32 (Eq. 3-4, v' = q - mu_g).
// A = z in three parts, block-diagonal over the item's distinct grains (row i
// holds its z at K = u RN .. u RN + RN - 1, u its slot's distinct grain, zeros
// elsewhere; only the K steps of the nd distinct grains run); B = those
// grains' basis parts for 64 coordinates, TMA boxes read MN-major. TMEM lane i,
// column t then holds (U^T z)_t of pair i (leading and cross products in two
// accumulators, as in the projection).
//   warp 0     TMA producer: per chunk, three parts of each slot's box.
//   warp 1     one thread issues the six part products into one of two
//              TMEM accumulators.
//   warps 2-9  epilogue: warp w reads lane quarter w % 4 (32 pairs), columns
//              32 (w - 2) / 4 .. + 31 of each chunk, and adds
//              ((q - mu) - U^T z)^2 from its pair's FP32 query row and the
//              grain's FP32 centre; it also writes the A operand of each item
//              before the item's MMAs.
template <int RN>
__global__ void __launch_bounds__(kR3Thr, 1) k_resid_tc3(
    const float* __restrict__ Q, const float* __restrict__ M, const __grid_constant__ CUtensorMap mapU3, int G,
    int d, int r, const uint4* __restrict__ slots, const uint32_t* __restrict__ n_slots,
    const uint32_t* __restrict__ pair_q, const float* __restrict__ zq, float* __restrict__ rhoq,
    int* __restrict__ err) {
  using P = ResidTc3<RN>;
  static_assert(P::kK % 64 == 0, "A rows are whole 128-byte swizzle atoms");
  constexpr int S = P::kStages;
  constexpr uint32_t kIdesc = tc::idesc_f32acc_bmn(1u, kPTM, kR3Chunk);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;                                // [part][K atom][128 rows x 128 B]
  uint8_t* sB = smem + kP3Parts * P::kBytesApart;    // [stage][part][slot][RN rows x 128 B]
  __shared__ __align__(8) uint64_t full[S], empty[S], accf[2], acce[2], afull, fin;
  __shared__ uint4 sslot[kPSlots];
  __shared__ float sred[kPTM];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  __shared__ uint32_t s_it_prod, s_it_mma;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 1) tc::tmem_alloc(&tmem_base, 4 * kR3Chunk);  // two chunks x (leading, cross)
  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
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
  // The basis ring and A start at zero: rows r .. RN - 1 of every box stay
  // zero (TMA writes r rows); a slot without pairs multiplies its stale or
  // zero box by zeros of A, which must be finite; A stays zero outside each
  // row's own slot range for good.
  for (uint32_t e = tid; e < (uint32_t)(S * P::kStage / 16); e += kR3Thr)
    *reinterpret_cast<uint4*>(sB + (size_t)e * 16) = make_uint4(0, 0, 0, 0);
  for (uint32_t e = tid; e < (uint32_t)(kP3Parts * P::kBytesApart / 16); e += kR3Thr)
    *reinterpret_cast<uint4*>(sA + (size_t)e * 16) = make_uint4(0, 0, 0, 0);
  tc::fence_proxy_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t ns = *n_slots;
  const uint32_t total = (ns + kPSlots - 1) / kPSlots;
  const int nch = (d + kR3Chunk - 1) / kR3Chunk;
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
        const uint32_t bytes = (uint32_t)(ig.nd * kP3Parts * r * 128);
        for (int c = 0; c < nch; ++c, ++it) {
          const int s = (int)(it % S);
          if (it >= (uint32_t)S && !tc::mbar_wait(&empty[s], ((it / S) - 1) & 1)) {
            ok = false;
            break;
          }
          uint8_t* st = sB + s * P::kStage;
          tc::mbar_expect_tx(&full[s], bytes);
#pragma unroll
          for (int p = 0; p < kP3Parts; ++p)
#pragma unroll
            for (int u = 0; u < kPSlots; ++u)
              if (u < ig.nd)
                tc::tma_load_2d(&mapU3, &full[s], st + p * P::kBytesBpart + u * P::kBytesBox, c * kR3Chunk,
                                p * G * r + (int)ig.grain(sl, u) * r);
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
      constexpr int kKS = P::kK / 16;
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
          const int s = (int)(it % S), a = (int)(ci & 1);
          if (ci >= 2 && !tc::mbar_wait(&acce[a], ((ci >> 1) - 1) & 1)) {
            ok = false;
            break;
          }
          if (!tc::mbar_wait(&full[s], (it / S) & 1)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t acc = tmem + (uint32_t)(a * 2 * kR3Chunk);  // leading products; cross at + kR3Chunk
          const uint32_t sbs = tc::smem_u32(sB + s * P::kStage);
          const uint32_t sa0 = tc::smem_u32(sA);
#pragma unroll
          for (int q = 0; q < kP3Prod; ++q)
#pragma unroll
            for (int ks = 0; ks < kKS; ++ks)
              if (ks < nks)
              tc::mma<true>(q == 0 ? acc : acc + (uint32_t)kR3Chunk,
                            tc::desc_sw128(sa0 + p3_a(q) * P::kBytesApart + (ks / 4) * (kPTM * 128) + (ks % 4) * 32),
                            tc::desc_sw128_mn(sbs + p3_b(q) * P::kBytesBpart + (ks / (RN / 16)) * P::kBytesBox +
                                                  (ks % (RN / 16)) * 2048,
                                              RN * 128),
                            kIdesc, ks != 0 || q > 1);
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
    const int et = tid - 64;            // 0 .. 255
    const int q4 = warp & 3;            // TMEM lane quarter = slot
    const int half = (warp - 2) >> 2;   // 0: columns 0..31 of a chunk, 1: 32..63
    const int row = q4 * 32 + lane;     // A row = TMEM lane = pair of the item
    bool failed = false;
    uint32_t li = 0, ci = 0;
    // this thread's A row (two threads per row, RN / 2 of its values each),
    // loaded for the next item while the current one runs
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
      if (zn_have) {
        // the row's K range is its slot's distinct grain's: u RN .. u RN + RN - 1
        uint4 slw[kPSlots];
#pragma unroll
        for (int j = 0; j < kPSlots; ++j) slw[j] = slot_of(w, j);
        const ItemGrains igw = item_grains(slw);
        int ua = 0;
#pragma unroll
        for (int j = 0; j < kPSlots; ++j)
          if (j == sa) ua = igw.u_of[j];
        if (prev_u >= 0 && prev_u != ua) {  // the range written last stays zero from now on
#pragma unroll
          for (int c8 = 0; c8 < kH / 8; ++c8) {
            const int kc = (prev_u * RN + hf * kH) / 8 + c8;
#pragma unroll
            for (int p = 0; p < kP3Parts; ++p)
              *reinterpret_cast<uint4*>(sA + p * P::kBytesApart + (kc / 8) * (kPTM * 128) +
                                        sw128_off(ra, (kc % 8) * 16)) = make_uint4(0, 0, 0, 0);
          }
        }
        prev_u = ua;
#pragma unroll
        for (int c8 = 0; c8 < kH / 8; ++c8) {  // 16-byte pieces of 8 values
          float v8[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) v8[u] = zn[c8 * 8 + u];
          uint4 parts[kP3Parts];
          split3_pack(v8, parts);
          const int kc = (ua * RN + hf * kH) / 8 + c8;  // piece index along K
#pragma unroll
          for (int p = 0; p < kP3Parts; ++p)
            *reinterpret_cast<uint4*>(sA + p * P::kBytesApart + (kc / 8) * (kPTM * 128) + sw128_off(ra, (kc % 8) * 16)) =
                parts[p];
        }
      }
      tc::fence_proxy_async_smem();
      tc::named_bar(1, 256);
      if (et == 0) tc::mbar_arrive(&afull);
      if (w + gridDim.x < total) prefetch_z(w + gridDim.x);
      const uint4 sl = sslot[q4];
      const bool mine = (uint32_t)lane < sl.z;
      const float* qrow = Q + (size_t)(mine ? pair_q[sl.y + lane] : 0u) * d;
      const float* mrow = M + (size_t)sl.x * d;
      float acc = 0.f;
      // this lane's 32 coordinates of a chunk, loaded one chunk ahead
      float4 qn[8];
      auto load_q = [&](int c) {
        const int t = c * kR3Chunk + half * 32;
#pragma unroll
        for (int g = 0; g < 8; ++g)
          qn[g] = (mine && c < nch && t + 4 * g < d) ? __ldg(reinterpret_cast<const float4*>(qrow + t + 4 * g))
                                                     : make_float4(0.f, 0.f, 0.f, 0.f);
      };
      load_q(0);
      for (int c = 0; c < nch; ++c, ++ci) {
        const int a = (int)(ci & 1);
        float4 qv[8];
#pragma unroll
        for (int g = 0; g < 8; ++g) qv[g] = qn[g];
        load_q(c + 1);
        if (!failed && __any_sync(0xffffffffu, !tc::mbar_wait(&accf[a], (ci >> 1) & 1))) failed = true;
        if (failed) continue;
        tc::fence_after_sync();
        float v[32], x[32];  // leading plus cross products
        const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(a * 2 * kR3Chunk + half * 32);
        tc::tmem_ld32(taddr, v);
        tc::tmem_ld32(taddr + kR3Chunk, x);
#pragma unroll
        for (int col = 0; col < 32; ++col) v[col] += x[col];
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&acce[a]);
        if (mine) {
          const int t0 = c * kR3Chunk + half * 32;
#pragma unroll
          for (int g = 0; g < 8; ++g) {
            if (t0 + 4 * g >= d) continue;  // past d: q = mu = reconstruction = 0
            const float4 m = __ldg(reinterpret_cast<const float4*>(mrow + t0 + 4 * g));
            const float e0 = (qv[g].x - m.x) - v[4 * g], e1 = (qv[g].y - m.y) - v[4 * g + 1];
            const float e2 = (qv[g].z - m.z) - v[4 * g + 2], e3 = (qv[g].w - m.w) - v[4 * g + 3];
            acc = fmaf(e0, e0, acc);
            acc = fmaf(e1, e1, acc);
            acc = fmaf(e2, e2, acc);
            acc = fmaf(e3, e3, acc);
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
    for (uint32_t q = s_it_mma; q < s_it_prod; ++q) tc::mbar_wait(&full[q % S], (q / S) & 1, 1u << 16);
  }
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 4 * kR3Chunk);
  }
  if (tid == 0 && s_fail) atomicOr(err, tc::kErrTimeout);
}

// The three BF16 parts of n FP32 values: out[p n + i] is part p of x[i].
__global__ void k_split3_bf16(const float* __restrict__ x, size_t n, uint16_t* __restrict__ out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float v = x[i];
#pragma unroll
    for (int p = 0; p < kP3Parts; ++p) {
      const uint16_t h = bf16_bits(v);
      out[(size_t)p * n + i] = h;
      v -= bf16_val(h);
    }
  }
}

}  // namespace
}  // namespace hntl
