// Centroid routing kernels (sec. 2.1 step 1, sec. 2.3 item 1): FP32
// direct-form distances to every centre, then the nprobe nearest by
// (distance, grain). Shared by the search path and the allocation-free
// routing entry point.
#pragma once

#include "hntl_internal.cuh"

namespace hntl {
namespace {

// ------------------------------------------------------------------ routing

constexpr int kRT = 64, kRK = 32;

// dist[q][g] = sum_t (Q[q][t] - M[g][t])^2 over a 64 x 64 tile; 256 threads,
// 4 x 4 outputs per thread; K staged through shared memory 32 columns at a time.
__global__ void __launch_bounds__(256) k_route_dist(const float* __restrict__ Q, const float* __restrict__ M, int nq,
                                                    int G, int d, float* __restrict__ dist) {
  __shared__ __align__(16) float sQ[kRK][kRT + 4];
  __shared__ __align__(16) float sM[kRK][kRT + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int q0 = blockIdx.y * kRT, g0 = blockIdx.x * kRT;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < d; k0 += kRK) {
#pragma unroll
    for (int i = 0; i < (kRT * kRK) / 256; ++i) {
      int e = threadIdx.x + 256 * i;
      int row = e / kRK, col = e % kRK;
      int q = q0 + row, g = g0 + row, t = k0 + col;
      sQ[col][row] = (q < nq && t < d) ? Q[(size_t)q * d + t] : 0.f;
      sM[col][row] = (g < G && t < d) ? M[(size_t)g * d + t] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kRK; ++kk) {
      float4 a = *reinterpret_cast<const float4*>(&sQ[kk][ty * 4]);
      float4 b = *reinterpret_cast<const float4*>(&sM[kk][tx * 4]);
      float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float t = av[i] - bv[j];
          acc[i][j] = fmaf(t, t, acc[i][j]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int q = q0 + ty * 4 + i;
    if (q >= nq) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int g = g0 + tx * 4 + j;
      if (g < G) dist[(size_t)q * G + g] = acc[i][j];
    }
  }
}

__device__ __forceinline__ bool lex_less(float a, int ia, float b, int ib) { return a < b || (a == b && ia < ib); }

// One warp per query: the query's G distances are staged in shared memory,
// then nprobe rounds each take the smallest (dist, g) above the previous one.
constexpr int kSelWarps = 4;
__global__ void __launch_bounds__(kSelWarps * 32) k_route_select(const float* __restrict__ dist, int nq, int G,
                                                                 int nprobe, int32_t* __restrict__ probe,
                                                                 float* __restrict__ probe_d) {
  extern __shared__ float sdist[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.x * kSelWarps + warp;
  if (q >= nq) return;
  float* row = sdist + (size_t)warp * G;
  for (int g = lane; g < G; g += 32) row[g] = dist[(size_t)q * G + g];
  __syncwarp();
  float pd = -INFINITY;
  int pg = -1;
  for (int p = 0; p < nprobe; ++p) {
    float bd = INFINITY;
    int bg = 0x7FFFFFFF;
    for (int g = lane; g < G; g += 32) {
      float x = row[g];
      if (!(x == x)) x = INFINITY;  // NaN (from a NaN query) sorts last, so every round still finds a grain
      if (lex_less(pd, pg, x, g) && lex_less(x, g, bd, bg)) {
        bd = x;
        bg = g;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float od = __shfl_xor_sync(0xffffffffu, bd, o);
      int og = __shfl_xor_sync(0xffffffffu, bg, o);
      if (lex_less(od, og, bd, bg)) {
        bd = od;
        bg = og;
      }
    }
    if (lane == 0) {
      probe[(size_t)q * nprobe + p] = bg;
      probe_d[(size_t)q * nprobe + p] = bd;
    }
    pd = bd;
    pg = bg;
  }
}

}  // namespace
}  // namespace hntl
