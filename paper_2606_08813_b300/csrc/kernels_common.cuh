// Kernels shared by the search path and the index builder.
#pragma once

#include <cuda_bf16.h>

#include "hntl_internal.cuh"

namespace hntl {
namespace {

constexpr int kPairsPerGroup = 8;  // (row, grain) pairs sharing one pass over a basis in k_project

// Block-wide exclusive scan of one value per thread (1024 threads).
template <typename T>
__device__ T block_exclusive_scan(T v, T* tot, T* warp_sums) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = lane < nw ? warp_sums[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) warp_sums[lane] = w;
    if (lane == nw - 1) *tot = w;
  }
  __syncthreads();
  T base = warp > 0 ? warp_sums[warp - 1] : T(0);
  T r = base + x - v;
  __syncthreads();
  return r;
}

// ------------------------------------------------------------------ projection

// One CTA per group of up to 8 (query, grain) pairs of one grain:
//   v' = q - mu_g (Eq. 1), z = U_g v' (Eq. 2), e = v' - U_g^T z (Eq. 3), rho_q = ||e||^2 (Eq. 4).
// The basis rows are read once per group and applied to all its pairs.
// kBF16 (precision form): q rounded to BF16, centres and bases read as BF16
// (Mv/Uv point to uint16 codes), arithmetic in FP32.
template <bool kBF16>
__device__ __forceinline__ float ld_val(const void* p, size_t i) {
  if (kBF16) return __uint_as_float((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p) + i) << 16);
  return __ldg(reinterpret_cast<const float*>(p) + i);
}

template <bool kBF16>
__global__ void __launch_bounds__(256) k_project(const float* __restrict__ Q, const void* __restrict__ Mv,
                                                 const void* __restrict__ Uv, int d, int r, int G,
                                                 const uint32_t* __restrict__ grp_off,
                                                 const uint32_t* __restrict__ pair_off,
                                                 const uint32_t* __restrict__ pair_q, float* __restrict__ zq,
                                                 float* __restrict__ rhoq) {
  extern __shared__ float sv[];  // [kPairsPerGroup][d]
  __shared__ float sz[kPairsPerGroup][kMaxR];
  __shared__ float sred[kPairsPerGroup][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t total = grp_off[G];
  for (uint32_t w = blockIdx.x; w < total; w += gridDim.x) {
    int lo = 0, hi = G;  // largest g with grp_off[g] <= w
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (grp_off[mid] <= w) lo = mid;
      else hi = mid;
    }
    const int g = lo;
    const uint32_t p0 = pair_off[g] + (w - grp_off[g]) * kPairsPerGroup;
    const int np = (int)min((uint32_t)kPairsPerGroup, pair_off[g + 1] - p0);
    const size_t mu0 = (size_t)g * d;
    for (int e = threadIdx.x; e < kPairsPerGroup * d; e += blockDim.x) {
      int p = e / d, t = e - p * d;
      float qv = 0.f;
      if (p < np) {
        qv = Q[(size_t)pair_q[p0 + p] * d + t];
        if (kBF16) qv = __bfloat162float(__float2bfloat16_rn(qv));
      }
      sv[e] = p < np ? qv - ld_val<kBF16>(Mv, mu0 + t) : 0.f;
    }
    __syncthreads();
    const size_t u0 = (size_t)g * r * d;
    for (int j = warp; j < r; j += 8) {
      float acc[kPairsPerGroup];
#pragma unroll
      for (int p = 0; p < kPairsPerGroup; ++p) acc[p] = 0.f;
      for (int t = lane; t < d; t += 32) {
        float u = ld_val<kBF16>(Uv, u0 + (size_t)j * d + t);
#pragma unroll
        for (int p = 0; p < kPairsPerGroup; ++p) acc[p] = fmaf(u, sv[p * d + t], acc[p]);
      }
#pragma unroll
      for (int p = 0; p < kPairsPerGroup; ++p) {
        float x = acc[p];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sz[p][j] = x;
      }
    }
    __syncthreads();
    float acc2[kPairsPerGroup];
#pragma unroll
    for (int p = 0; p < kPairsPerGroup; ++p) acc2[p] = 0.f;
    for (int t = threadIdx.x; t < d; t += blockDim.x) {
      float e[kPairsPerGroup];
#pragma unroll
      for (int p = 0; p < kPairsPerGroup; ++p) e[p] = sv[p * d + t];
      for (int j = 0; j < r; ++j) {
        float u = ld_val<kBF16>(Uv, u0 + (size_t)j * d + t);
#pragma unroll
        for (int p = 0; p < kPairsPerGroup; ++p) e[p] = fmaf(-sz[p][j], u, e[p]);
      }
#pragma unroll
      for (int p = 0; p < kPairsPerGroup; ++p) acc2[p] = fmaf(e[p], e[p], acc2[p]);
    }
#pragma unroll
    for (int p = 0; p < kPairsPerGroup; ++p) {
      float x = acc2[p];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) sred[p][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < np) {
      int p = threadIdx.x;
      float s = 0.f;
#pragma unroll
      for (int i = 0; i < 8; ++i) s += sred[p][i];
      rhoq[p0 + p] = s;
    }
    for (int e = threadIdx.x; e < np * r; e += blockDim.x) {
      int p = e / r, j = e - p * r;
      zq[(size_t)(p0 + p) * r + j] = sz[p][j];
    }
    __syncthreads();
  }
}

// Bitonic sort of n (a power of two) 64-bit keys in shared memory.
__device__ void bitonic_sort_u64(unsigned long long* a, int n) {
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int ixj = i ^ j;
        if (ixj > i) {
          unsigned long long x = a[i], y = a[ixj];
          bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ int pow2_at_least(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

// The bin of a histogram holding the need-th smallest (1-based) element, and
// how many elements lie in lower bins. All threads call it.
__device__ void find_bin(const uint32_t* hist, int nbins, uint32_t need, uint32_t* s_bin, uint32_t* s_below,
                         uint32_t* scratch) {
  const int per = (nbins + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per;
  uint32_t sum = 0;
  for (int i = 0; i < per && b0 + i < nbins; ++i) sum += hist[b0 + i];
  uint32_t excl = block_exclusive_scan<uint32_t>(sum, scratch + 64, scratch);
  if (excl < need && excl + sum >= need) {
    uint32_t run = excl;
    for (int i = 0; i < per && b0 + i < nbins; ++i) {
      uint32_t h = hist[b0 + i];
      if (run + h >= need) {
        *s_bin = (uint32_t)(b0 + i);
        *s_below = run;
        break;
      }
      run += h;
    }
  }
  __syncthreads();
}

}  // namespace
}  // namespace hntl
