// General BF16 GEMM on tcgen05 for the learned router: C[M x N] = A[M x K] B[N x K]^T
// (both operands K-major BF16, FP32 accumulation in TMEM), 128 x BN tiles
// (BN = 128, or 64 where 128-wide tiles would leave SMs idle), operands
// streamed by TMA through a 3-stage ring (two or more CTAs per SM, so one
// CTA's epilogue overlaps another's main loop). The epilogue adds an
// optional bias over N, writes the FP32 result (the pre-activation) and,
// optionally, a BF16 copy of it or of its exact (erf) GELU; each warp's
// 32 x 32 pieces go through shared memory so that rows are stored whole.
#pragma once

#include <cuda_bf16.h>

#include "hntl_internal.cuh"
#include "tc_common.cuh"

namespace hntl {
namespace {

constexpr int kGTM = 128, kGTN = 128, kGStages = 3;  // 96 KB of stages at BN = 128: two CTAs per SM
template <int BN>
constexpr int gemm_smem() {
  return kGStages * (kGTM + BN) * 128 + 1024;
}

struct GemmEpi {
  float* C;            // [M][ldc] FP32, or nullptr
  uint16_t* Cb;        // [M][ldc] BF16 of the activation, or nullptr
  const float* bias;   // [N], or nullptr
  int gelu;            // Cb = bf16(gelu(C)) instead of bf16(C)
  int ldc;
};

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

template <int BN>
__global__ void __launch_bounds__(128, 2) k_gemm_tn(const __grid_constant__ CUtensorMap mapA,
                                                 const __grid_constant__ CUtensorMap mapB, int M, int N, int K,
                                                 GemmEpi epi, int* __restrict__ err) {
  constexpr int kKB = 64;  // BF16 elements per stage (128-byte rows)
  static_assert(BN == 64 || BN == 128, "tile width");
  constexpr uint32_t kBytesA = kGTM * 128, kBytesB = BN * 128;
  constexpr uint32_t kIdesc = tc::idesc_f32acc(1u, kGTM, BN);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kGStages], empty[kGStages], done;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::tmem_alloc(&tmem_base, BN);
  if (tid == 32) {
    for (int s = 0; s < kGStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(&done, 1);
    tc::mbar_fence_init();
    s_fail = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const int m0 = blockIdx.y * kGTM, n0 = blockIdx.x * BN;
  const int nkb = (K + kKB - 1) / kKB;
  // The producer and the MMA issuer are lane 0 of warps 0 and 1; the other
  // lanes of those warps wait at __syncwarp (not on an mbarrier poll, which
  // would hold the whole warp, the working lane included, between polls).
  if (warp == 0) {
    if (lane == 0) {
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % kGStages;
        if (kb >= kGStages && !tc::mbar_wait(&empty[s], ((kb / kGStages) - 1) & 1)) {
          atomicExch(&s_fail, 1);
          break;
        }
        uint8_t* sa = smem + s * (kBytesA + kBytesB);
        tc::mbar_expect_tx(&full[s], kBytesA + kBytesB);
        tc::tma_load_2d(&mapA, &full[s], sa, kb * kKB, m0);
        tc::tma_load_2d(&mapB, &full[s], sa + kBytesA, kb * kKB, n0);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % kGStages;
        if (!tc::mbar_wait(&full[s], (kb / kGStages) & 1)) {
          atomicExch(&s_fail, 1);
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t sa = tc::smem_u32(smem + s * (kBytesA + kBytesB));
#pragma unroll
        for (int ks = 0; ks < kKB / 16; ++ks)
          tc::mma<true>(tmem, tc::desc_sw128(sa + ks * 32), tc::desc_sw128(sa + kBytesA + ks * 32), kIdesc,
                        (kb | ks) != 0);
        tc::mma_commit(&empty[s]);
      }
      if (ok) tc::mma_commit(&done);
    }
    __syncwarp();
  }
  const bool waited = tc::mbar_wait(&done, 0);
  const bool failed = __syncthreads_or(!waited || s_fail);
  tc::fence_after_sync();
  if (!failed) {
    // every MMA has completed and every stage was consumed: the stage memory is free
    float* tile = reinterpret_cast<float*>(smem) + warp * 32 * 33;  // this warp's 32 x 32 piece, padded
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      float v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c0, v);  // lane = row
#pragma unroll
      for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = v[j];
      __syncwarp();
      const int col = n0 + c0 + lane;  // lane = column from here
      const float b = (epi.bias && col < N) ? epi.bias[col] : 0.f;
#pragma unroll 4
      for (int i = 0; i < 32; ++i) {
        const int row = m0 + warp * 32 + i;
        if (row < M && col < N) {
          const float pre = epi.bias ? tile[i * 33 + lane] + b : tile[i * 33 + lane];
          const size_t o = (size_t)row * epi.ldc + col;
          if (epi.C) epi.C[o] = pre;
          if (epi.Cb) epi.Cb[o] = __bfloat16_as_ushort(__float2bfloat16_rn(epi.gelu ? gelu_f(pre) : pre));
        }
      }
      __syncwarp();
    }
  } else if (tid == 0) {
    atomicOr(err, tc::kErrTimeout);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, BN);
}

}  // namespace
}  // namespace hntl
