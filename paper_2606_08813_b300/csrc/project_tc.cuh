// Query projection on the tensor cores for the precision form (Eq. 1-4 with
// BF16 query, centres and bases).
//
// One CTA per (grain g, up to 128 of its pairs). Two A operands per K step:
// the pairs' BF16 query rows q_b and the grain's centre row -mu_b repeated on
// every row; the B operand is the grain's BF16 basis U_g (r rows, K-major).
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

constexpr int kPTM = 128;                 // pairs per item (MMA M)
constexpr int kPGroup = kPTM;             // pairs per work item
constexpr int kPKB = 64;                  // BF16 elements per K block (128 bytes)
constexpr uint32_t kPBytesA = kPTM * 128; // one A operand per K block
template <int RN>
struct ProjTc {
  static constexpr uint32_t kBytesB = RN * 128;
  static constexpr uint32_t kStage = 2 * kPBytesA + kBytesB;
  static constexpr int kSmem = 2 * kStage + 1024;
};

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_val(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// swizzled byte offset of (row, byte) in a K-major 128B-swizzled tile
__device__ __forceinline__ uint32_t sw128_off(int row, int byte) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((byte >> 4) ^ (row & 7)) << 4) | (byte & 15)));
}

// RN = basis rows padded to a multiple of 16 (MMA N), r <= RN.
template <int RN>
__global__ void __launch_bounds__(128) k_project_tc(const uint16_t* __restrict__ Qh, const uint16_t* __restrict__ Mh,
                                                    const uint16_t* __restrict__ Uh, const float* __restrict__ gram,
                                                    int d, int r, int G, int nprobe,
                                                    const uint32_t* __restrict__ grp_off,
                                                    const uint32_t* __restrict__ pair_off,
                                                    const uint32_t* __restrict__ pair_q,
                                                    const uint32_t* __restrict__ pair_p,
                                                    const float* __restrict__ probe_d, float* __restrict__ zq,
                                                    float* __restrict__ rhoq, int* __restrict__ err) {
  using P = ProjTc<RN>;
  constexpr uint32_t kIdesc = tc::idesc_f32acc(1u, kPTM, RN);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ float sgram[RN * RN];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) tc::tmem_alloc(&tmem_base, RN < 32 ? 32 : RN);
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::mbar_fence_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  uint32_t phase[2] = {0, 0};
  bool failed = false;
  const uint32_t total = grp_off[G];
  const int nkb = (d + kPKB - 1) / kPKB;
  for (uint32_t w = blockIdx.x; w < total && !failed; w += gridDim.x) {
    int lo = 0, hi = G;  // largest g with grp_off[g] <= w
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (grp_off[mid] <= w) lo = mid;
      else hi = mid;
    }
    const int g = lo;
    const uint32_t p0 = pair_off[g] + (w - grp_off[g]) * kPGroup;
    const int np = (int)min((uint32_t)kPGroup, pair_off[g + 1] - p0);
    for (int e = tid; e < RN * RN; e += 128) {
      const int a = e / RN, b = e % RN;
      sgram[e] = (a < r && b < r) ? gram[((size_t)g * r + a) * r + b] : 0.f;
    }
    const bool has_row = tid < np;
    const uint16_t* qrow = has_row ? Qh + (size_t)pair_q[p0 + tid] * d : nullptr;
    const uint16_t* mrow = Mh + (size_t)g * d;
    for (int kb = 0; kb < nkb; ++kb) {
      const int s = kb & 1;
      uint8_t* st = smem + s * P::kStage;
      if (kb >= 2) {  // the MMAs that read this buffer two K blocks ago must be done
        if (!tc::mbar_wait(&bar[s], phase[s])) failed = true;
        phase[s] ^= 1;
      }
      if (__syncthreads_or(failed)) {
        failed = true;
        break;
      }
      // A operands: this thread's query row and the negated centre, 128 bytes each
      // (rows past the last pair are left as they are: their accumulators are never read)
      const int k0 = kb * kPKB;
      if (has_row) {
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
          const int kk = k0 + ch * 8;
          uint4 qv = make_uint4(0, 0, 0, 0), mv = make_uint4(0, 0, 0, 0);
          if (kk + 8 <= d) {
            qv = __ldg(reinterpret_cast<const uint4*>(qrow + kk));
            mv = __ldg(reinterpret_cast<const uint4*>(mrow + kk));
          }
          mv.x ^= 0x80008000u;  // -mu: flip both BF16 sign bits
          mv.y ^= 0x80008000u;
          mv.z ^= 0x80008000u;
          mv.w ^= 0x80008000u;
          const uint32_t off = sw128_off(tid, ch * 16);
          *reinterpret_cast<uint4*>(st + off) = qv;
          *reinterpret_cast<uint4*>(st + kPBytesA + off) = mv;
        }
      }
      // B: basis rows of grain g (rows >= r are zero)
      uint8_t* sb = st + 2 * kPBytesA;
      for (int e = tid; e < RN * 8; e += 128) {  // 8 chunks of 16 bytes per row
        const int row = e >> 3, ch = e & 7;
        uint4 v = make_uint4(0, 0, 0, 0);
        const int kk = k0 + ch * 8;
        if (row < r) {
          const uint16_t* src = Uh + ((size_t)g * r + row) * d + kk;
          if (kk + 8 <= d) {
            v = *reinterpret_cast<const uint4*>(src);
          } else {
            uint16_t tmp[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int i = 0; i < 8 && kk + i < d; ++i) tmp[i] = src[i];
            v = *reinterpret_cast<const uint4*>(tmp);
          }
        }
        *reinterpret_cast<uint4*>(sb + sw128_off(row, ch * 16)) = v;
      }
      tc::fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
        const uint32_t sa = tc::smem_u32(st);
#pragma unroll
        for (int ks = 0; ks < kPKB / 16; ++ks)
#pragma unroll
          for (int part = 0; part < 2; ++part)  // + U q_b, then - U mu_b, over the same 16 coordinates
            tc::mma<true>(tmem, tc::desc_sw128(sa + part * kPBytesA + ks * 32),
                          tc::desc_sw128(sa + 2 * kPBytesA + ks * 32), kIdesc, (kb | ks | part) != 0);
        tc::mma_commit(&bar[s]);
      }
    }
    if (failed) break;
    // drain: the last commit of each buffer still in flight
    for (int s = 0; s < 2 && s < nkb; ++s) {
      if (!tc::mbar_wait(&bar[s], phase[s])) failed = true;
      phase[s] ^= 1;
    }
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }
    tc::fence_after_sync();
    // epilogue: warp w owns TMEM lanes 32w..32w+31 = pair rows
    float z[RN];
#pragma unroll
    for (int c0 = 0; c0 < RN; c0 += 32) {
      float v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (c0 + j < RN) z[c0 + j] = v[j];
    }
    if (has_row) {
      float zz = 0.f, qf = 0.f;
#pragma unroll
      for (int a = 0; a < RN; ++a) {
        if (a >= r) break;
        zz = fmaf(z[a], z[a], zz);
        float row = 0.f;
#pragma unroll
        for (int b = 0; b < RN; ++b)
          if (b < r) row = fmaf(sgram[a * RN + b], z[b], row);
        qf = fmaf(z[a], row, qf);
      }
      const uint32_t pr = p0 + tid;
      const float vnorm = probe_d[(size_t)pair_q[pr] * nprobe + pair_p[pr]];
      const float rho = (vnorm - 2.f * zz) + qf;
      rhoq[p0 + tid] = rho > 0.f ? rho : 0.f;
      float* out = zq + (size_t)(p0 + tid) * r;
#pragma unroll
      for (int a = 0; a < RN; ++a)
        if (a < r) out[a] = z[a];
    }
    tc::fence_before_sync();
    __syncthreads();  // TMEM and sgram are reused by the next item
    tc::fence_after_sync();
  }
  if (failed && tid == 0) atomicOr(err, tc::kErrTimeout);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, RN < 32 ? 32 : RN);
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
