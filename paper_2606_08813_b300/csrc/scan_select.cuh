// Block-SoA scan (Eq. 6) fused with the pool of the C best (Table 1, "Pool C").
//
// Three kernels replace "write every distance, then select":
//   k_pilot        one CTA per query computes D for max(1024, 4C) rows, at
//                  most 2048 (whole Block-SoA blocks, evenly spaced), of its
//                  nearest probed grains in routing order and takes the C-th
//                  smallest as tau_q. Those are real rows of the query's
//                  probe set, so at least C rows have D <= tau_q and tau_q is
//                  an upper bound on the query's true C-th distance. tau_q is
//                  taken to 16 bits (two radix passes) and rounded up to the
//                  top of that bin: still a bound, at most 2^-7 looser.
//   k_scan_filter  grain-major scan of every probed Block-SoA block: a
//                  grain's coordinates are read once and applied to every
//                  query that probes it; rows with D <= tau_q (and passing
//                  the query's attribute range) are appended to the query's
//                  survivor list as (D, id) keys. Since D >= rho_q + rho_i,
//                  and rounding is monotone, a (query, block) pair with
//                  fl(rho_q + min rho_i over the block) > tau_q has no
//                  survivor and is skipped; a block no pair needs is not read.
//   k_final_select one CTA per query: the exact C smallest (D, id) of the
//                  survivors, or, if the survivors overflowed their buffer,
//                  of all probed rows recomputed on the fly (same result).
// D is computed by one function everywhere (eval_D; eval_D_i16 in the
// 16-bit form), so a row's D is bitwise the same in the pilot, the scan and
// the fallback.
#pragma once

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "hntl_internal.cuh"
#include "kernels_common.cuh"

namespace hntl {
namespace {

constexpr int kPilotRows = 2048;  // most rows the pilot evaluates per query (whole 128-row blocks)
constexpr int kPilotMin = 1024;   // fewest (when 4 C is smaller)
constexpr int kTieCap = 1024;
constexpr uint32_t kInfBits = 0x7F800000u;

__host__ __device__ inline uint32_t survivor_cap(uint32_t C) { return C * 32 > 16384 ? C * 32 : 16384; }

__device__ __forceinline__ unsigned long long pack2(float a, float b) {
  return ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(a);
}

// D = ||z_q - z_i||^2 + rho_q + rho_i with packed FP32x2 arithmetic: even and
// odd coordinates accumulate in two lanes (each lane rounds exactly like
// fmaf), then the lanes are added and the residual norms appended. zq may
// point to shared or global memory (8-byte aligned, RT floats, zero padded).
template <int RT>
__device__ __forceinline__ float eval_D(const float* zq, const float (&z)[RT], float rho_q, float rho_i) {
  unsigned long long acc = 0ull;
#pragma unroll
  for (int j = 0; j < RT; j += 2) {
    const unsigned long long q2 = *reinterpret_cast<const unsigned long long*>(zq + j);
    const unsigned long long z2 = pack2(z[j], z[j + 1]);
    unsigned long long df;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(df) : "l"(q2), "l"(z2));
    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(acc) : "l"(df), "l"(acc));
  }
  const float s = __uint_as_float((uint32_t)acc) + __uint_as_float((uint32_t)(acc >> 32));
  return (s + rho_q) + rho_i;
}

// The r coordinates of row t of block b into registers (zero padded to RT):
// FP32 values, or FP8-E4M3 codes decoded exactly (through half precision) and
// multiplied by the grain scale in FP32.
struct Coords {
  const float* Zb;      // FP32 form
  const uint8_t* Z8b;   // precision form
  const float* scale;   // precision form (FP8 scale) and 16-bit form (coordinate step), per grain
  const int16_t* Z16b;  // 16-bit form
};

template <int RT, int kC>
__device__ __forceinline__ void load_row(const Coords& c, int rp, float s_g, size_t b, int t, float (&z)[RT]) {
  if constexpr (kC == kCoordFP8) {
    static_assert(RT % 16 == 0, "FP8 rows are read in lanes of 16 codes");
#pragma unroll
    for (int l = 0; l < RT / 16; ++l) {
      if (l * 16 < rp) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(c.Z8b + ((b * (rp / 16) + l) * kBlockRows + t) * 16));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const float2 a = __half22float2(
              __half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[h] & 0xFFFFu), __NV_E4M3)));
          const float2 e = __half22float2(
              __half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[h] >> 16), __NV_E4M3)));
          z[l * 16 + 4 * h + 0] = a.x * s_g;
          z[l * 16 + 4 * h + 1] = a.y * s_g;
          z[l * 16 + 4 * h + 2] = e.x * s_g;
          z[l * 16 + 4 * h + 3] = e.y * s_g;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) z[l * 16 + i] = 0.f;
      }
    }
  } else if constexpr (kC == kCoordI16) {
    // 16-bit form: 8 int16 codes per lane, times the grain's step (the code is exact in FP32)
    static_assert(RT % 8 == 0, "16-bit rows are read in lanes of 8 codes");
#pragma unroll
    for (int l = 0; l < RT / 8; ++l) {
      if (l * 8 < rp) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(c.Z16b + ((b * (rp / 8) + l) * kBlockRows + t) * 8));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          z[l * 8 + 2 * h] = (float)(int16_t)(w[h] & 0xFFFFu) * s_g;
          z[l * 8 + 2 * h + 1] = (float)(int16_t)(w[h] >> 16) * s_g;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) z[l * 8 + i] = 0.f;
      }
    }
  } else {
#pragma unroll
    for (int l = 0; l < RT / 4; ++l) {
      if (l * 4 < rp) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(c.Zb + ((b * (rp / 4) + l) * kBlockRows + t) * 4));
        z[4 * l] = v.x;
        z[4 * l + 1] = v.y;
        z[4 * l + 2] = v.z;
        z[4 * l + 3] = v.w;
      } else {
        z[4 * l] = z[4 * l + 1] = z[4 * l + 2] = z[4 * l + 3] = 0.f;
      }
    }
  }
}

// ------------------------------------------------------------------ 16-bit form: integer Eq. 6

// The 16-bit form evaluates Eq. 6 on the codes themselves (Eq. 5 states the
// integer representations the scan works on): with the query's codes q_j, a
// row's codes c_j (both on the grain's step delta_g) and their residuals on
// the grain's residual grid,
//   S = sum_j (q_j - c_j)^2 = |q|^2 + |c|^2 - 2 q.c     (exact in integers)
//   D = fl32(fl32(delta_g^2) * fl32(S)) + fl32(rho_q + rho_i)
// in IEEE single precision with separate roundings. q.c runs on the integer
// dot-product units: a row word holds two int16 codes, and dp2a multiplies
// them by two 8-bit pieces of the query codes, so each query code is split as
// q = 256 hi + lo (hi signed, lo unsigned) and q.c = 256 (c.hi) + (c.lo), each
// partial sum within int32 (|c| <= 16383 by the row steps, |hi| <= 128,
// lo <= 255, r <= 64). |c|^2 uses the same split of the row's own codes.
__device__ __forceinline__ int dp2a_lo_ss(uint32_t a, uint32_t b, int c) {
  int d;
  asm("dp2a.lo.s32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ int dp2a_hi_ss(uint32_t a, uint32_t b, int c) {
  int d;
  asm("dp2a.hi.s32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ int dp2a_lo_su(uint32_t a, uint32_t b, int c) {
  int d;
  asm("dp2a.lo.s32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ int dp2a_hi_su(uint32_t a, uint32_t b, int c) {
  int d;
  asm("dp2a.hi.s32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// A row of the 16-bit form: its codes, two per word (word m = codes 2m, 2m+1,
// the lower code in the low half), zero past rp.
template <int RT>
__device__ __forceinline__ void i16_load_row(const int16_t* __restrict__ Z16b, int rp, size_t b, int t,
                                             uint32_t (&w)[RT / 2]) {
  static_assert(RT % 8 == 0, "16-bit rows are read in lanes of 8 codes");
#pragma unroll
  for (int l = 0; l < RT / 8; ++l) {
    uint4 v = make_uint4(0, 0, 0, 0);
    if (l * 8 < rp) v = __ldg(reinterpret_cast<const uint4*>(Z16b + ((b * (rp / 8) + l) * kBlockRows + t) * 8));
    w[4 * l] = v.x;
    w[4 * l + 1] = v.y;
    w[4 * l + 2] = v.z;
    w[4 * l + 3] = v.w;
  }
}

// |c|^2 of a row's codes: per word, its high bytes (signed) and low bytes
// (unsigned) gathered by byte permutes, two dp2a.
template <int RT>
__device__ __forceinline__ long long i16_row_norm(const uint32_t (&w)[RT / 2]) {
  int ah = 0, al = 0;
#pragma unroll
  for (int m = 0; m < RT / 2; ++m) {
    ah = dp2a_lo_ss(w[m], __byte_perm(w[m], 0u, 0x0031u), ah);
    al = dp2a_lo_su(w[m], __byte_perm(w[m], 0u, 0x0020u), al);
  }
  return 256ll * ah + al;
}

// The query side of one (query, grain) pair: high and low bytes of its codes,
// four codes per word (word m = codes 4m .. 4m+3), |q|^2 and its residual.
template <int RT>
struct I16Query {
  uint32_t hi[RT / 4];
  uint32_t lo[RT / 4];
  long long qn;
  float rho;
};

// Packs codes[0 .. r) (zero past r) into hi/lo byte words.
template <int RT>
__device__ __forceinline__ void i16_pack_query(const int16_t* __restrict__ codes, int r, uint32_t* hi, uint32_t* lo) {
#pragma unroll
  for (int m = 0; m < RT / 4; ++m) {
    uint32_t h = 0, l = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int j = 4 * m + e;
      const int c = j < r ? (int)codes[j] : 0;
      h |= (uint32_t)((c >> 8) & 0xFF) << (8 * e);
      l |= (uint32_t)(c & 0xFF) << (8 * e);
    }
    hi[m] = h;
    lo[m] = l;
  }
}

// The 16-bit form's per-pair query codes (workspace, written by the
// quantisation step): codes [pairs][rp] int16 (zero past r) and |q|^2 [pairs].
// Null in the other forms.
struct I16Pairs {
  const int16_t* codes;
  const long long* qn;
};

// D of a (pair, row) of the 16-bit form, bitwise the same wherever it is
// evaluated (pilot, scan, pool fallback).
template <int RT>
__device__ __forceinline__ float eval_D_i16(const uint32_t* hi, const uint32_t* lo, long long qn, float rho_q,
                                            const uint32_t (&w)[RT / 2], long long ni, float rho_i, float dl2) {
  int ah = 0, al = 0;
#pragma unroll
  for (int m = 0; m < RT / 4; ++m) {
    const uint32_t h = hi[m], l = lo[m];
    ah = dp2a_lo_ss(w[2 * m], h, ah);
    ah = dp2a_hi_ss(w[2 * m + 1], h, ah);
    al = dp2a_lo_su(w[2 * m], l, al);
    al = dp2a_hi_su(w[2 * m + 1], l, al);
  }
  const long long S = qn + ni - 2 * (256ll * ah + al);
  return __fadd_rn(__fmul_rn(dl2, __ll2float_rn(S)), __fadd_rn(rho_q, rho_i));
}

// ------------------------------------------------------------------ block interval bound

// Rows are laid out in each grain by their first coordinate, so a block's
// decoded first coordinates span a short interval [lo, hi]. For a row of the
// block, D >= (z_q0 - z_i0)^2 + rho_q + rho_i >= gap^2 + rho_q + min rho, with
// gap the distance from z_q0 to the interval; the scan's FP32 D is at least
// (1 - 2^-18) of that exact value, so with a 2^-16 margin on the left a block
// for which this returns true has no row with D <= tau (the survivors are the
// same as without the bound).
__device__ __forceinline__ bool interval_prunes(float zq0, float2 iv, float rho_q, float rmin, float tau) {
  const float gap = fmaxf(fmaxf(iv.x - zq0, zq0 - iv.y), 0.f);
  return (rho_q + rmin + gap * gap) * (1.f - 0x1p-16f) > tau;
}

// [min, max] of the decoded first coordinate of each block's real rows
// ([+inf, -inf] for a block without rows), one CTA of 128 threads per block.
template <int RT, int kC>
__global__ void __launch_bounds__(kBlockRows) k_block_z0(const Coords cz, const uint32_t* __restrict__ blk_grain,
                                                         const uint32_t* __restrict__ blk_off,
                                                         const uint32_t* __restrict__ grain_rows, int rp,
                                                         float2* __restrict__ out) {
  __shared__ float s_lo[4], s_hi[4];
  const size_t b = blockIdx.x;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const uint32_t g = blk_grain[b];
  const bool valid = (uint32_t)(b - blk_off[g]) * kBlockRows + t < grain_rows[g];
  float z[RT];
  load_row<RT, kC>(cz, rp, kC != kCoordF32 ? cz.scale[g] : 1.f, b, t, z);
  float lo = valid ? z[0] : INFINITY, hi = valid ? z[0] : -INFINITY;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if (lane == 0) {
    s_lo[warp] = lo;
    s_hi[warp] = hi;
  }
  __syncthreads();
  if (t == 0)
    out[b] = make_float2(fminf(fminf(s_lo[0], s_lo[1]), fminf(s_lo[2], s_lo[3])),
                         fmaxf(fmaxf(s_hi[0], s_hi[1]), fmaxf(s_hi[2], s_hi[3])));
}

// ------------------------------------------------------------------ pilot

template <int RT, int kC>
__global__ void __launch_bounds__(256) k_pilot(int nprobe, int C, const int32_t* __restrict__ probe,
                                               const uint32_t* __restrict__ pair_of,
                                               const uint32_t* __restrict__ blk_off,
                                               const uint32_t* __restrict__ grain_rows, const Coords cz,
                                               const float* __restrict__ rho, const int64_t* __restrict__ attr_b,
                                               int r, int rp, const float* __restrict__ zq,
                                               const float* __restrict__ rhoq, const int64_t* __restrict__ filter,
                                               float* __restrict__ tau, const uint32_t* __restrict__ qC,
                                               const I16Pairs q16) {
  __shared__ uint32_t vals[kPilotRows];  // D bit patterns (non-negative floats order like unsigned)
  __shared__ uint32_t hist[256];
  __shared__ __align__(8) float szq[RT];
  __shared__ uint32_t s16hi[RT / 4 > 0 ? RT / 4 : 1], s16lo[RT / 4 > 0 ? RT / 4 : 1];
  __shared__ long long s16qn;
  __shared__ uint32_t scratch[96];
  __shared__ uint32_t s_fill, s_bin, s_below, s_total;
  const int q = blockIdx.x;
  if (qC) C = (int)qC[q];  // per-query pool size (mixed batches)
  // rows to evaluate: enough that the C-th smallest is a useful bound (a larger
  // sample only tightens tau, which costs more here than it saves downstream)
  const uint32_t budget = (uint32_t)min(kPilotRows, max(kPilotMin, 4 * C));
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) s_fill = 0;
  long long lo = 0, hi = 0;
  if (filter) {
    lo = filter[2 * (size_t)q];
    hi = filter[2 * (size_t)q + 1];
  }
  uint32_t scanned = 0;  // rows evaluated so far (block-uniform)
  for (int p = 0; p < nprobe; ++p) {
    __syncthreads();
    const uint32_t fill = s_fill;
    if (fill >= (uint32_t)C) break;
    // unfiltered: `budget` rows in all; filtered: whole blocks until `budget` rows
    // passed the range (the buffer holds kPilotRows), scanning at most 8 kPilotRows
    if (!filter && scanned + kBlockRows > budget) break;
    if (filter && (fill >= budget || fill + kBlockRows > (uint32_t)kPilotRows ||
                   scanned + kBlockRows > 8u * kPilotRows))
      break;
    const int g = probe[(size_t)q * nprobe + p];
    const uint32_t s = pair_of[(size_t)q * nprobe + p];
    const uint32_t n = grain_rows[g];
    const uint32_t nbk = blk_off[g + 1] - blk_off[g];
    for (int j = threadIdx.x; j < RT; j += blockDim.x) szq[j] = j < r ? zq[(size_t)s * r + j] : 0.f;
    if constexpr (kC == kCoordI16) {
      if (threadIdx.x == 0) {
        i16_pack_query<RT>(q16.codes + (size_t)s * rp, r, s16hi, s16lo);
        s16qn = q16.qn[s];
      }
    }
    const float rho_q = rhoq[s];
    const float s_g = kC != kCoordF32 ? cz.scale[g] : 1.f;
    __syncthreads();
    const uint32_t room = filter ? min(((uint32_t)kPilotRows - fill) / kBlockRows,
                                       (8u * kPilotRows - scanned) / kBlockRows)
                                 : (budget - scanned) / kBlockRows;
    const uint32_t take = nbk < room ? nbk : room;  // whole blocks, evenly spaced over the grain
    for (uint32_t e0 = 0; e0 < take * kBlockRows; e0 += blockDim.x) {  // block-uniform trip count
      const uint32_t e = e0 + threadIdx.x;
      bool keep = false;
      uint32_t k = 0;
      if (e < take * kBlockRows) {
        const uint32_t i = e / kBlockRows;
        const int t = e % kBlockRows;
        const uint32_t jb = take == nbk ? i : (uint32_t)(((unsigned long long)i * nbk) / take);
        const size_t b = blk_off[g] + jb;
        keep = jb * kBlockRows + t < n;
        if (keep && filter) {
          const long long a = attr_b[b * kBlockRows + t];
          keep = a >= lo && a <= hi;
        }
        if (keep) {
          if constexpr (kC == kCoordI16) {
            uint32_t w[RT / 2];
            i16_load_row<RT>(cz.Z16b, rp, b, t, w);
            k = __float_as_uint(eval_D_i16<RT>(s16hi, s16lo, s16qn, rho_q, w, i16_row_norm<RT>(w),
                                               rho[b * kBlockRows + t], __fmul_rn(s_g, s_g)));
          } else {
            float z[RT];
            load_row<RT, kC>(cz, rp, s_g, b, t, z);
            k = __float_as_uint(eval_D<RT>(szq, z, rho_q, rho[b * kBlockRows + t]));
          }
          keep = k < kInfBits;
        }
      }
      // one shared-memory atomic per warp for the slots of its kept rows
      const unsigned mask = __ballot_sync(0xffffffffu, keep);
      uint32_t base = 0;
      if (lane == 0 && mask) base = atomicAdd(&s_fill, (uint32_t)__popc(mask));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (keep) vals[base + __popc(mask & ((1u << lane) - 1u))] = k;
    }
    scanned += take * kBlockRows;
  }
  __syncthreads();
  const uint32_t fill = s_fill;
  if (fill < (uint32_t)C) {
    if (threadIdx.x == 0) tau[q] = INFINITY;
    return;
  }
  // the C-th smallest of vals[0..fill) to its top 16 bits (two 8-bit radix
  // digits); tau_q is the top of that bin, at most 2^-7 relative above the
  // C-th smallest value, so still an upper bound on the query's true C-th
  // distance (the pool is selected exactly downstream; a looser tau only
  // admits a few more survivors)
  uint32_t prefix = 0, need = (uint32_t)C;
  int known = 0;
  for (int pass = 0; pass < 2; ++pass) {
    const int sh = 24 - 8 * pass;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < fill; i += blockDim.x) {
      const uint32_t k = vals[i];
      if (known && (k >> (32 - known)) != prefix) continue;
      atomicAdd(&hist[(k >> sh) & 255u], 1u);
    }
    __syncthreads();
    find_bin(hist, 256, need, &s_bin, &s_below, scratch);
    need -= s_below;
    prefix = (prefix << 8) | s_bin;
    known += 8;
    __syncthreads();
  }
  (void)s_total;
  if (threadIdx.x == 0) tau[q] = __uint_as_float((prefix << 16) | 0xFFFFu);  // finite: every value is below +inf
}

// ------------------------------------------------------------------ scan

constexpr int kMaxNeed = 1024;  // pairs of one grain a block can list after pruning

template <int RT, int kC>
__global__ void __launch_bounds__(kBlockRows, 8) k_scan_filter(
    const uint32_t* __restrict__ blk_grain, const uint32_t* __restrict__ blk_off,
    const uint32_t* __restrict__ grain_rows, const Coords cz, const float* __restrict__ rho,
    const uint32_t* __restrict__ ids, const int64_t* __restrict__ attr_b, int r, int rp,
    const uint32_t* __restrict__ gcnt, const uint32_t* __restrict__ pair_off, const uint32_t* __restrict__ pair_q,
    const float* __restrict__ zq, const float* __restrict__ rhoq, const float* __restrict__ tau,
    const float* __restrict__ blk_rho_min, const float2* __restrict__ blk_z0, const int64_t* __restrict__ filter,
    uint32_t cap, uint32_t* __restrict__ cnt, unsigned long long* __restrict__ surv, const I16Pairs q16) {
  constexpr int kChunk = 32;
  constexpr bool kI = kC == kCoordI16;
  __shared__ __align__(8) float sz[kI ? 1 : kChunk][kI ? 2 : RT];
  __shared__ uint32_t s16hi[kI ? kChunk : 1][kI ? RT / 4 : 1], s16lo[kI ? kChunk : 1][kI ? RT / 4 : 1];
  __shared__ long long s16qn[kI ? kChunk : 1];
  __shared__ float srho[kChunk], stau[kChunk];
  __shared__ uint32_t sq[kChunk];
  __shared__ long long slo[kChunk], shi[kChunk];
  __shared__ uint32_t s_need[kMaxNeed];
  __shared__ uint32_t s_nneed;
  const size_t b = blockIdx.x;
  const uint32_t g = blk_grain[b];
  const uint32_t m = gcnt[g];
  if (m == 0) return;
  const int t = threadIdx.x, lane = t & 31;
  const uint32_t p_begin = pair_off[g];
  const float rmin = blk_rho_min[b];
  // the pairs of this grain that can still reach their pool from this block
  if (t == 0) s_nneed = 0;
  __syncthreads();
  const float2 iv = blk_z0[b];
  for (uint32_t s = t; s < m; s += kBlockRows) {
    const float rq = rhoq[p_begin + s], tq = tau[pair_q[p_begin + s]];
    if (rq + rmin <= tq && !interval_prunes(zq[(size_t)(p_begin + s) * r], iv, rq, rmin, tq)) {
      const uint32_t pos = atomicAdd(&s_nneed, 1u);
      if (pos < (uint32_t)kMaxNeed) s_need[pos] = s;
    }
  }
  __syncthreads();
  const uint32_t nneed = s_nneed;
  if (nneed == 0) return;
  const bool listed = nneed <= (uint32_t)kMaxNeed;  // else walk every pair and test each
  const uint32_t nwalk = listed ? nneed : m;
  const uint32_t row = (uint32_t)(b - blk_off[g]) * kBlockRows + t;
  const bool valid = row < grain_rows[g];
  float z[kI ? 1 : RT];
  uint32_t w16[kI ? RT / 2 : 1];
  long long ni = 0;
  float dl2 = 0.f;
  if constexpr (kI) {
    i16_load_row<RT>(cz.Z16b, rp, b, t, w16);
    ni = i16_row_norm<RT>(w16);
    const float dl = cz.scale[g];
    dl2 = __fmul_rn(dl, dl);
  } else {
    load_row<RT, kC>(cz, rp, kC != kCoordF32 ? cz.scale[g] : 1.f, b, t, z);
  }
  const float rho_i = rho[b * kBlockRows + t];
  const uint32_t id = ids[b * kBlockRows + t];
  const long long a = filter ? (long long)attr_b[b * kBlockRows + t] : 0;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (uint32_t s0 = 0; s0 < nwalk; s0 += kChunk) {
    const int ns = (int)min((uint32_t)kChunk, nwalk - s0);
    if constexpr (!kI) {
      for (int e = t; e < kChunk * RT; e += kBlockRows) {
        const int s = e / RT, j = e - s * RT;
        float v = 0.f;
        if (s < ns && j < r) {
          const uint32_t pr = p_begin + (listed ? s_need[s0 + s] : s0 + s);
          v = zq[(size_t)pr * r + j];
        }
        sz[s][j] = v;
      }
    }
    if (t < ns) {
      const uint32_t pr = p_begin + (listed ? s_need[s0 + t] : s0 + t);
      if constexpr (kI) {
        i16_pack_query<RT>(q16.codes + (size_t)pr * rp, r, s16hi[t], s16lo[t]);
        s16qn[t] = q16.qn[pr];
      }
      const uint32_t q = pair_q[pr];
      sq[t] = q;
      srho[t] = rhoq[pr];
      stau[t] = tau[q];
      if (filter) {
        slo[t] = (long long)filter[2 * (size_t)q];
        shi[t] = (long long)filter[2 * (size_t)q + 1];
      }
    }
    __syncthreads();
    for (int s = 0; s < ns; ++s) {
      if (srho[s] + rmin > stau[s]) continue;  // no row of this block can reach the query's pool
      float D;
      if constexpr (kI) D = eval_D_i16<RT>(s16hi[s], s16lo[s], s16qn[s], srho[s], w16, ni, rho_i, dl2);
      else D = eval_D<RT>(&sz[s][0], z, srho[s], rho_i);
      const bool ok = valid && D <= stau[s] && (!filter || (a >= slo[s] && a <= shi[s]));
      const unsigned mask = __ballot_sync(0xffffffffu, ok);
      if (mask) {
        const int leader = __ffs(mask) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(&cnt[sq[s]], (uint32_t)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (ok) {
          const uint32_t pos = base + __popc(mask & lt_mask);
          if (pos < cap)
            surv[(size_t)sq[s] * cap + pos] = ((unsigned long long)__float_as_uint(D) << 32) | id;
        }
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ selection

// Elements as (D bit pattern, id): the survivor list of one query.
struct SurvivorSrc {
  const unsigned long long* keys;
  uint32_t n;
  template <class F>
  __device__ void for_each(F f) const {
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      const unsigned long long k = keys[i];
      f((uint32_t)(k >> 32), (uint32_t)(k & 0xFFFFFFFFu));
    }
  }
};

// Elements as (D bit pattern, id): every row of the query's probed grains,
// D recomputed (used when the survivor list overflowed).
template <int RT, int kC>
struct ProbedRowsSrc {
  int q, nprobe, r, rp;
  const int32_t* probe;
  const uint32_t* pair_of;
  const uint32_t* blk_off;
  const uint32_t* grain_rows;
  Coords cz;
  const float* rho;
  const uint32_t* ids;
  const int64_t* attr_b;
  const float* zq;
  const float* rhoq;
  const int64_t* filter;
  I16Pairs q16;
  template <class F>
  __device__ void for_each(F f) const {
    long long lo = 0, hi = 0;
    if (filter) {
      lo = filter[2 * (size_t)q];
      hi = filter[2 * (size_t)q + 1];
    }
    for (int p = 0; p < nprobe; ++p) {
      const int g = probe[(size_t)q * nprobe + p];
      const uint32_t s = pair_of[(size_t)q * nprobe + p];
      const uint32_t n = grain_rows[g];
      const float rho_q = rhoq[s];
      const float s_g = kC != kCoordF32 ? cz.scale[g] : 1.f;
      if constexpr (kC == kCoordI16) {
        uint32_t qh[RT / 4], ql[RT / 4];
        i16_pack_query<RT>(q16.codes + (size_t)s * rp, r, qh, ql);
        const long long qn = q16.qn[s];
        const float dl2 = __fmul_rn(s_g, s_g);
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
          const size_t b = blk_off[g] + i / kBlockRows;
          const int t = i % kBlockRows;
          if (filter) {
            const long long a = attr_b[b * kBlockRows + t];
            if (a < lo || a > hi) continue;
          }
          uint32_t w[RT / 2];
          i16_load_row<RT>(cz.Z16b, rp, b, t, w);
          f(__float_as_uint(eval_D_i16<RT>(qh, ql, qn, rho_q, w, i16_row_norm<RT>(w), rho[b * kBlockRows + t], dl2)),
            ids[b * kBlockRows + t]);
        }
      } else {
        __align__(8) float zl[RT];
#pragma unroll
        for (int j = 0; j < RT; ++j) zl[j] = j < r ? zq[(size_t)s * r + j] : 0.f;
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
          const size_t b = blk_off[g] + i / kBlockRows;
          const int t = i % kBlockRows;
          if (filter) {
            const long long a = attr_b[b * kBlockRows + t];
            if (a < lo || a > hi) continue;
          }
          float z[RT];
          load_row<RT, kC>(cz, rp, s_g, b, t, z);
          f(__float_as_uint(eval_D<RT>(zl, z, rho_q, rho[b * kBlockRows + t])), ids[b * kBlockRows + t]);
        }
      }
    }
  }
};

constexpr int kSelDigits = 4, kSelBits = 8;  // radix select on the D bit pattern, 8 bits at a time
constexpr int kSelBinCap = 256;              // bin size below which two digits suffice
constexpr int kSelRankMax = 256;             // pool size up to which the output is ordered by counting

struct SelSmem {
  uint32_t hist[1 << kSelBits];
  unsigned long long keys[kMaxC];
  unsigned long long tk[kTieCap];
  uint32_t scratch[96];
  uint32_t s_bin, s_below, s_total, s_nout, s_nties, s_min;
};

// The exact C smallest (D, id) of a source, written sorted to out_id/out_d
// (pads: id 0xFFFFFFFF, +inf). Four 8-bit radix digits of the D bit pattern
// find the C-th smallest D; ties at that D are resolved by the smaller ids.
template <class Src>
__device__ void select_topc(const Src& src, int C, SelSmem& S, uint32_t* __restrict__ out_id,
                            float* __restrict__ out_d) {
  uint32_t prefix = 0, need = (uint32_t)C;
  int known = 0;
  bool take_all = false, short_bin = false;
  for (int pass = 0; pass < kSelDigits; ++pass) {
    const int nb = 1 << kSelBits;
    const int sh = 32 - kSelBits * (pass + 1);
    for (int i = threadIdx.x; i < nb; i += blockDim.x) S.hist[i] = 0;
    __syncthreads();
    const int kn = known;
    const uint32_t pf = prefix;
    src.for_each([&](uint32_t k, uint32_t) {
      if (k >= kInfBits) return;
      if (kn && (k >> (32 - kn)) != pf) return;
      atomicAdd(&S.hist[(k >> sh) & (nb - 1)], 1u);
    });
    __syncthreads();
    if (pass == 0) {
      uint32_t sum = 0;
      for (int i = threadIdx.x; i < nb; i += blockDim.x) sum += S.hist[i];
      block_exclusive_scan<uint32_t>(sum, &S.s_total, S.scratch);
      if (S.s_total <= need) {
        take_all = true;
        break;
      }
    }
    find_bin(S.hist, nb, need, &S.s_bin, &S.s_below, S.scratch);
    need -= S.s_below;
    prefix = (prefix << kSelBits) | S.s_bin;
    known += kSelBits;
    // after two digits the bin holding the C-th key is usually small: finish
    // by ordering that bin's keys instead of two more passes over the source
    const bool small_bin = pass == 1 && S.hist[S.s_bin] <= (uint32_t)kSelBinCap;  // block-uniform
    __syncthreads();
    if (small_bin) {
      short_bin = true;
      break;
    }
  }
  if (threadIdx.x == 0) {
    S.s_nout = 0;
    S.s_nties = 0;
  }
  __syncthreads();
  uint32_t nout;
  if (short_bin) {
    // keys whose top 16 bits are below the bin's are in the pool; the bin's
    // keys (at most kSelBinCap) are ranked by (D, id) and the first `need` kept
    const uint32_t T16 = prefix;
    src.for_each([&](uint32_t k, uint32_t id) {
      if (k >= kInfBits) return;
      const unsigned long long key = ((unsigned long long)k << 32) | id;
      if ((k >> 16) < T16) S.keys[atomicAdd(&S.s_nout, 1u)] = key;
      else if ((k >> 16) == T16) S.tk[atomicAdd(&S.s_nties, 1u)] = key;
    });
    __syncthreads();
    const uint32_t nb_ = S.s_nout, nt = S.s_nties;
    for (uint32_t i = threadIdx.x; i < nt; i += blockDim.x) {
      const unsigned long long me = S.tk[i];
      uint32_t rank = 0;
      for (uint32_t j = 0; j < nt; ++j) rank += S.tk[j] < me ? 1u : 0u;
      if (rank < need) S.keys[nb_ + rank] = me;
    }
    nout = (uint32_t)C;
  } else {
  const uint32_t T = take_all ? kInfBits : prefix;
  src.for_each([&](uint32_t k, uint32_t id) {
    if (k >= kInfBits) return;
    if (k < T) {
      const uint32_t pos = atomicAdd(&S.s_nout, 1u);
      if (pos < (uint32_t)kMaxC) S.keys[pos] = ((unsigned long long)k << 32) | id;
    } else if (k == T) {
      const uint32_t pos = atomicAdd(&S.s_nties, 1u);
      if (pos < (uint32_t)kTieCap) S.tk[pos] = id;
    }
  });
  __syncthreads();
  nout = S.s_nout;
  if (!take_all) {
    const uint32_t need_eq = (uint32_t)C - nout;
    if (S.s_nties <= (uint32_t)kTieCap) {
      const int nt = (int)S.s_nties;
      const int np2 = pow2_at_least(nt);
      for (int i = threadIdx.x; i < np2; i += blockDim.x)
        if (i >= nt) S.tk[i] = ~0ull;
      __syncthreads();
      bitonic_sort_u64(S.tk, np2);
      for (uint32_t i = threadIdx.x; i < need_eq; i += blockDim.x)
        S.keys[nout + i] = ((unsigned long long)T << 32) | (uint32_t)S.tk[i];
    } else {
      // more ties than the buffer: take the smallest remaining id, need_eq times
      uint32_t last = 0;
      bool first = true;
      for (uint32_t e = 0; e < need_eq; ++e) {
        if (threadIdx.x == 0) S.s_min = 0xFFFFFFFFu;
        __syncthreads();
        uint32_t mine = 0xFFFFFFFFu;
        const bool fst = first;
        const uint32_t lst = last;
        src.for_each([&](uint32_t k, uint32_t id) {
          if (k == T && (fst || id > lst) && id < mine) mine = id;
        });
        atomicMin(&S.s_min, mine);
        __syncthreads();
        last = S.s_min;
        first = false;
        if (threadIdx.x == 0) S.keys[nout + e] = ((unsigned long long)T << 32) | last;
        __syncthreads();
      }
    }
    nout = (uint32_t)C;
  }
  }
  __syncthreads();
  // output in (D, id) order. Up to kSelRankMax keys: the keys are distinct
  // (each id once), so a key's position is the number of smaller keys (no
  // barriers); more: a bitonic sort (its cost grows as n log^2 n, the count's
  // as n^2)
  if (nout <= (uint32_t)kSelRankMax) {
    for (uint32_t i = threadIdx.x; i < nout; i += blockDim.x) {
      const unsigned long long me = S.keys[i];
      uint32_t rank = 0;
      for (uint32_t j = 0; j < nout; ++j) rank += S.keys[j] < me ? 1u : 0u;
      out_id[rank] = (uint32_t)(me & 0xFFFFFFFFu);
      out_d[rank] = __uint_as_float((uint32_t)(me >> 32));
    }
  } else {
    const int n2 = pow2_at_least((int)nout);
    for (int i = threadIdx.x; i < n2; i += blockDim.x)
      if (i >= (int)nout) S.keys[i] = ~0ull;
    __syncthreads();
    bitonic_sort_u64(S.keys, n2);
    for (uint32_t i = threadIdx.x; i < nout; i += blockDim.x) {
      const unsigned long long kk = S.keys[i];
      out_id[i] = (uint32_t)(kk & 0xFFFFFFFFu);
      out_d[i] = __uint_as_float((uint32_t)(kk >> 32));
    }
  }
  for (int i = (int)nout + threadIdx.x; i < C; i += blockDim.x) {
    out_id[i] = kInvalidId;
    out_d[i] = INFINITY;
  }
}

constexpr int kFinalThreads = 128;  // small CTAs: many queries in flight per SM

// The pool from the survivors (kFallback = false: one CTA per query), or, for
// the queries whose survivors overflowed their buffer, from every probed row
// recomputed (kFallback = true: a small grid; each CTA checks 128 queries at
// a time and selects for the overflowed ones, which are rare). A CTA of the
// common kernel returns at once for an overflowed query. Keeping the rare
// recompute out of the common kernel keeps its registers low, and its
// occupancy high.
template <int RT, int kC, bool kFallback>
__global__ void __launch_bounds__(kFinalThreads, kFallback ? 1 : 8) k_final_select(
    int nprobe, int C, uint32_t cap, const uint32_t* __restrict__ cnt, const unsigned long long* __restrict__ surv,
    const int32_t* __restrict__ probe, const uint32_t* __restrict__ pair_of, const uint32_t* __restrict__ blk_off,
    const uint32_t* __restrict__ grain_rows, const Coords cz, const float* __restrict__ rho,
    const uint32_t* __restrict__ ids, const int64_t* __restrict__ attr_b, int r, int rp,
    const float* __restrict__ zq, const float* __restrict__ rhoq, const int64_t* __restrict__ filter,
    uint32_t* __restrict__ cand_id, float* __restrict__ cand_d, const uint32_t* __restrict__ qC,
    const I16Pairs q16, uint32_t nq) {
  __shared__ SelSmem S;
  auto select_one = [&](int q) {
    const uint32_t n = cnt[q];
    uint32_t* oid = cand_id + (size_t)q * C;  // rows are C (the batch's largest pool) apart
    float* od = cand_d + (size_t)q * C;
    int Cq = C;
    if (qC) {  // mixed batch: this query's own pool size, the rest of its row padded
      Cq = (int)qC[q];
      for (int i = Cq + threadIdx.x; i < C; i += blockDim.x) {
        oid[i] = kInvalidId;
        od[i] = INFINITY;
      }
    }
    if constexpr (!kFallback) {
      SurvivorSrc src{surv + (size_t)q * cap, n};
      select_topc(src, Cq, S, oid, od);
    } else {
      ProbedRowsSrc<RT, kC> src{q,  nprobe, r,   rp,     probe, pair_of, blk_off, grain_rows,
                                  cz, rho,    ids, attr_b, zq,    rhoq,    filter,  q16};
      select_topc(src, Cq, S, oid, od);
    }
  };
  if constexpr (!kFallback) {
    const int q = blockIdx.x;
    if (cnt[q] > cap) return;
    select_one(q);
  } else {
    __shared__ uint32_t s_over[kFinalThreads];
    __shared__ uint32_t s_nover;
    for (uint32_t q0 = blockIdx.x * kFinalThreads; q0 < nq; q0 += gridDim.x * kFinalThreads) {
      if (threadIdx.x == 0) s_nover = 0;
      __syncthreads();
      const uint32_t qq = q0 + threadIdx.x;
      if (qq < nq && cnt[qq] > cap) s_over[atomicAdd(&s_nover, 1u)] = qq;
      __syncthreads();
      const uint32_t nover = s_nover;
      for (uint32_t i = 0; i < nover; ++i) {
        select_one((int)s_over[i]);
        __syncthreads();
      }
      __syncthreads();  // every thread has read s_nover before the next pass resets it
    }
  }
}

}  // namespace
}  // namespace hntl
