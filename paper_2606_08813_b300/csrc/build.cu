// GPU index builder: grain partition, per-grain local bases, database
// coordinates, Block-SoA layout (and the precision form's FP8/BF16 copies).
//
// The paper does not fix the partitioning (sec. 2.2 only asks for "spatial
// grains" with a centroid); this builder uses k-means++ seeding (Arthur and
// Vassilvitskii, 2007; the G uniform draws are an input) and Lloyd
// iterations on a strided training subset, then one assignment pass of all
// rows and exact means of the final members. The local basis of each grain
// (sec. 2.2, W_g) is the dominant r-dimensional invariant subspace of the
// grain's covariance, found by orthogonal (subspace) iteration: Y = C V,
// V = orth(Y) by two-pass modified Gram-Schmidt. Any orthonormal basis of
// that subspace gives the same distances (Eq. 6 is invariant under a rotation
// inside the subspace), so no Rayleigh-Ritz ordering is needed. Database
// coordinates and residual norms follow Eq. 1-4 with the same projection
// kernel the queries use.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "hntl_internal.cuh"
#include "kernels_common.cuh"

namespace hntl {

namespace {

// ------------------------------------------------------------------ nearest centre

constexpr int kNT = 64, kNK = 32;

// packed[i] = min over g of (bits(||x_i - m_g||^2) << 32 | g): the lexicographic
// (distance, grain) minimum. Distances are non-negative, so their bit patterns
// order like their values. 64 x 64 tile per CTA, 4 x 4 per thread.
template <bool kTile>
__global__ void __launch_bounds__(256) k_nearest(const float* __restrict__ X, int64_t n, const float* __restrict__ M,
                                                 int G, int d, unsigned long long* __restrict__ packed,
                                                 float* __restrict__ tile) {
  __shared__ __align__(16) float sX[kNK][kNT + 4];
  __shared__ __align__(16) float sM[kNK][kNT + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t q0 = (int64_t)blockIdx.y * kNT;
  const int g0 = blockIdx.x * kNT;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < d; k0 += kNK) {
#pragma unroll
    for (int i = 0; i < (kNT * kNK) / 256; ++i) {
      int e = threadIdx.x + 256 * i;
      int row = e / kNK, col = e % kNK;
      int64_t q = q0 + row;
      int g = g0 + row, t = k0 + col;
      sX[col][row] = (q < n && t < d) ? X[q * d + t] : 0.f;
      sM[col][row] = (g < G && t < d) ? M[(size_t)g * d + t] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kNK; ++kk) {
      float4 a = *reinterpret_cast<const float4*>(&sX[kk][ty * 4]);
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
  if constexpr (kTile) {  // every distance of the tile, rows of G (each sums t = 0 .. d-1 in order, by fmaf)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t q = q0 + ty * 4 + i;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int g = g0 + tx * 4 + j;
        if (q < n && g < G) tile[q * G + g] = acc[i][j];
      }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    unsigned long long best = ~0ull;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int g = g0 + tx * 4 + j;
      if (g < G) {
        float v = acc[i][j];
        if (!(v == v)) v = INFINITY;
        unsigned long long key = ((unsigned long long)__float_as_uint(v) << 32) | (uint32_t)g;
        best = key < best ? key : best;
      }
    }
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
      unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
      best = other < best ? other : best;
    }
    int64_t q = q0 + ty * 4 + i;
    if (tx == 0 && q < n && best != ~0ull) atomicMin(&packed[q], best);
  }
}

__global__ void k_unpack(const unsigned long long* __restrict__ packed, int64_t n, int32_t* __restrict__ assign,
                         float* __restrict__ dist, const int32_t* __restrict__ prev, unsigned int* __restrict__ changed) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long p = packed[i];
  int32_t g = (int32_t)(p & 0xFFFFFFFFu);
  assign[i] = g;
  if (dist) dist[i] = __uint_as_float((uint32_t)(p >> 32));
  if (prev && prev[i] != g) atomicAdd(changed, 1u);
}

// The K nearest centres of each of n rows (row i = X[rows[i]], or X[i] when
// rows is null) as ascending (distance bits << 32 | grain) keys: one CTA per
// 64-row block walks every 64-centre tile with k_nearest's arithmetic (so a
// distance is bitwise the one k_nearest forms), writes the tile's distances to
// shared memory, and the row's owner thread merges them into the row's sorted
// list (most values fail the list's current K-th key and are skipped).
template <int K>
__global__ void __launch_bounds__(256) k_nearest_topk(const float* __restrict__ X, const uint64_t* __restrict__ rows,
                                                      int64_t n, const float* __restrict__ M, int G, int d,
                                                      unsigned long long* __restrict__ out) {
  __shared__ __align__(16) float sX[kNK][kNT + 4];
  __shared__ __align__(16) float sM[kNK][kNT + 4];
  __shared__ float sD[kNT][kNT + 1];
  __shared__ unsigned long long sTop[kNT][K];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t q0 = (int64_t)blockIdx.x * kNT;
  for (int e = threadIdx.x; e < kNT * K; e += 256) sTop[e / K][e % K] = ~0ull;
  for (int g0 = 0; g0 < G; g0 += kNT) {
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < d; k0 += kNK) {
#pragma unroll
      for (int i = 0; i < (kNT * kNK) / 256; ++i) {
        const int e = threadIdx.x + 256 * i;
        const int row = e / kNK, col = e % kNK;
        const int64_t q = q0 + row;
        const int g = g0 + row, t = k0 + col;
        float xv = 0.f;
        if (q < n && t < d) xv = X[(rows ? (int64_t)rows[q] : q) * d + t];
        sX[col][row] = xv;
        sM[col][row] = (g < G && t < d) ? M[(size_t)g * d + t] : 0.f;
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < kNK; ++kk) {
        const float4 a = *reinterpret_cast<const float4*>(&sX[kk][ty * 4]);
        const float4 b = *reinterpret_cast<const float4*>(&sM[kk][tx * 4]);
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float t = av[i] - bv[j];
            acc[i][j] = fmaf(t, t, acc[i][j]);
          }
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) sD[ty * 4 + i][tx * 4 + j] = acc[i][j];
    __syncthreads();
    if (threadIdx.x < kNT && q0 + threadIdx.x < n) {
      unsigned long long* top = sTop[threadIdx.x];
      unsigned long long worst = top[K - 1];
      const int lim = min(kNT, G - g0);
      for (int c = 0; c < lim; ++c) {
        float v = sD[threadIdx.x][c];
        if (!(v == v)) v = INFINITY;
        const unsigned long long key = ((unsigned long long)__float_as_uint(v) << 32) | (uint32_t)(g0 + c);
        if (key >= worst) continue;
        int p = K - 1;  // insert, keeping the list sorted
        while (p > 0 && top[p - 1] > key) {
          top[p] = top[p - 1];
          --p;
        }
        top[p] = key;
        worst = top[K - 1];
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < kNT * K; e += 256) {
    const int64_t q = q0 + e / K;
    if (q < n) out[q * K + e % K] = sTop[e / K][e % K];
  }
}

// One warp per row of a distance tile [n][G]: its K smallest (distance, grain)
// keys in ascending order (K rounds of a warp minimum above the last pick).
__global__ void k_topk_rows(const float* __restrict__ tile, int64_t n, int G, int K,
                            unsigned long long* __restrict__ out) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const float* row = tile + w * G;
  unsigned long long last = 0;
  for (int k = 0; k < K; ++k) {
    unsigned long long best = ~0ull;
    for (int g = lane; g < G; g += 32) {
      float v = row[g];
      if (!(v == v)) v = INFINITY;
      const unsigned long long key = ((unsigned long long)__float_as_uint(v) << 32) | (uint32_t)g;
      if ((k == 0 || key > last) && key < best) best = key;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
      best = other < best ? other : best;
    }
    last = best;
    if (lane == 0) out[w * K + k] = best;
  }
}

// ------------------------------------------------------------------ k-means++ and means

// rows of X gathered by index into a contiguous buffer
__global__ void k_gather_rows(const float* __restrict__ X, const uint64_t* __restrict__ rows, int64_t n, int d,
                              float* __restrict__ out) {
  int64_t i = blockIdx.x;
  if (i >= n) return;
  const float* src = X + rows[i] * d;
  for (int t = threadIdx.x; t < d; t += blockDim.x) out[i * d + t] = src[t];
}

// warp per row: dmin = ||x - c||^2 (init) or min(dmin, ||x - c||^2)
__global__ void k_kpp_dist(const float* __restrict__ Xs, int64_t n, int d, const float* __restrict__ c,
                           float* __restrict__ dmin, int init) {
  int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= n) return;
  const float* x = Xs + w * d;
  float acc = 0.f;
  for (int t = lane; t < d; t += 32) {
    float df = x[t] - c[t];
    acc = fmaf(df, df, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) dmin[w] = init ? acc : fminf(dmin[w], acc);
}

// Single CTA: the smallest row i whose running sum of dmin exceeds u * total
// (FP64 sums); that row becomes centre c.
__global__ void __launch_bounds__(1024) k_kpp_pick(const float* __restrict__ dmin, int64_t n, double u,
                                                   const float* __restrict__ Xs, int d, float* __restrict__ Mc,
                                                   long long* __restrict__ chosen) {
  __shared__ double ws[32];
  __shared__ double s_tot;
  __shared__ long long s_pick;
  const int64_t per = (n + blockDim.x - 1) / blockDim.x;
  const int64_t b0 = (int64_t)threadIdx.x * per;
  double sum = 0.0;
  for (int64_t i = b0; i < b0 + per && i < n; ++i) sum += (double)dmin[i];
  if (threadIdx.x == 0) s_pick = -1;
  double excl = block_exclusive_scan<double>(sum, &s_tot, ws);
  const double total = s_tot;
  const double target = u * total;
  if (total > 0.0 && excl <= target && target < excl + sum) {
    double run = excl;
    long long pick = -1;
    for (int64_t i = b0; i < b0 + per && i < n; ++i) {
      run += (double)dmin[i];
      if (run > target) {
        pick = i;
        break;
      }
    }
    if (pick < 0) pick = (long long)min(n - 1, b0 + per - 1);
    atomicMax(&s_pick, pick);
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_pick < 0) {
    long long p = (long long)(u * (double)n);
    s_pick = p >= n ? n - 1 : p;
  }
  __syncthreads();
  const long long pick = s_pick;
  if (threadIdx.x == 0) *chosen = pick;
  for (int t = threadIdx.x; t < d; t += blockDim.x) Mc[t] = Xs[pick * d + t];
}

// warp per row: FP64 atomic sums of member rows and member counts
__global__ void k_accum(const float* __restrict__ X, int64_t n, int d, const int32_t* __restrict__ assign,
                        double* __restrict__ sums, unsigned int* __restrict__ counts) {
  int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= n) return;
  int g = assign[w];
  const float* x = X + w * d;
  double* s = sums + (size_t)g * d;
  for (int t = lane; t < d; t += 32) atomicAdd(s + t, (double)x[t]);
  if (lane == 0) atomicAdd(counts + g, 1u);
}

__global__ void k_means_finalize(const double* __restrict__ sums, const unsigned int* __restrict__ counts, int G,
                                 int d, float* __restrict__ M) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)G * d) return;
  int g = (int)(e / d);
  if (counts[g]) M[e] = (float)(sums[e] / (double)counts[g]);
}

// ------------------------------------------------------------------ local bases

constexpr int kCT = 64;

// Covariance of each grain, (1/n_g) sum (x - mu)(x - mu)^T, one 64 x 64
// lower-triangle tile per CTA (blockIdx.x = triangular tile index,
// blockIdx.y = grain within the batch), rows gathered by grain-ordered id,
// FP32 products over 32-row chunks added into FP64 accumulators.
__global__ void __launch_bounds__(256) k_cov(const float* __restrict__ X, const uint32_t* __restrict__ ids_g,
                                             const uint32_t* __restrict__ goff, const float* __restrict__ M, int d,
                                             int g0, float* __restrict__ C) {
  __shared__ __align__(16) float A[32][kCT + 4];
  __shared__ __align__(16) float B[32][kCT + 4];
  int ta = 0, rem = blockIdx.x;
  while (rem > ta) {
    rem -= ta + 1;
    ++ta;
  }
  const int tb = rem;  // tb <= ta
  const int g = g0 + blockIdx.y;
  const uint32_t start = goff[g], ng = goff[g + 1] - start;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const float* mu = M + (size_t)g * d;
  double accd[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) accd[i][j] = 0.0;
  for (uint32_t r0 = 0; r0 < ng; r0 += 32) {
#pragma unroll
    for (int i = 0; i < (32 * kCT) / 256; ++i) {
      int e = threadIdx.x + 256 * i;
      int row = e / kCT, col = e % kCT;
      float av = 0.f, bv = 0.f;
      if (r0 + row < ng) {
        const float* x = X + (size_t)ids_g[start + r0 + row] * d;
        int ca = ta * kCT + col, cb = tb * kCT + col;
        if (ca < d) av = x[ca] - mu[ca];
        if (cb < d) bv = x[cb] - mu[cb];
      }
      A[row][col] = av;
      B[row][col] = bv;
    }
    __syncthreads();
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 4
    for (int rr = 0; rr < 32; ++rr) {
      float4 a = *reinterpret_cast<const float4*>(&A[rr][ty * 4]);
      float4 b = *reinterpret_cast<const float4*>(&B[rr][tx * 4]);
      float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) accd[i][j] += (double)acc[i][j];
    __syncthreads();
  }
  const double inv = ng ? 1.0 / (double)ng : 0.0;
  float* Cg = C + (size_t)blockIdx.y * d * d;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int a = ta * kCT + ty * 4 + i;
    if (a >= d) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int b = tb * kCT + tx * 4 + j;
      if (b >= d) continue;
      float v = (float)(accd[i][j] * inv);
      Cg[(size_t)a * d + b] = v;
      Cg[(size_t)b * d + a] = v;
    }
  }
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// V[g][j][t] uniform in [-1, 1) from a counter-based hash (SplitMix64 finaliser)
__global__ void k_init_basis(float* __restrict__ V, int64_t n, unsigned long long seed) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  unsigned long long h = mix64(seed ^ mix64((unsigned long long)e));
  V[e] = (float)((double)(h >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
}

// Y[g][j][a] = sum_b C[g][a][b] V[g][j][b]: 64 output rows per CTA, all r columns.
template <int RT>
__global__ void __launch_bounds__(256) k_cov_apply(const float* __restrict__ C, const float* __restrict__ V,
                                                   int d, int r, float* __restrict__ Y) {
  __shared__ float Cs[kCT][kCT + 1];
  __shared__ float Vs[RT][kCT];
  const int g = blockIdx.y;
  const int a0 = blockIdx.x * kCT;
  const int al = threadIdx.x & 63, jg = threadIdx.x >> 6;  // jg in 0..3
  const float* Cg = C + (size_t)g * d * d;
  const float* Vg = V + (size_t)g * r * d;
  constexpr int kPer = RT / 4;
  float acc[kPer];
#pragma unroll
  for (int m = 0; m < kPer; ++m) acc[m] = 0.f;
  for (int b0 = 0; b0 < d; b0 += kCT) {
    for (int e = threadIdx.x; e < kCT * kCT; e += 256) {
      int ar = e / kCT, bc = e % kCT;
      int a = a0 + ar, b = b0 + bc;
      Cs[ar][bc] = (a < d && b < d) ? Cg[(size_t)a * d + b] : 0.f;
    }
    for (int e = threadIdx.x; e < RT * kCT; e += 256) {
      int j = e / kCT, bc = e % kCT;
      int b = b0 + bc;
      Vs[j][bc] = (j < r && b < d) ? Vg[(size_t)j * d + b] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int bb = 0; bb < kCT; ++bb) {
      float c = Cs[al][bb];
#pragma unroll
      for (int m = 0; m < kPer; ++m) acc[m] = fmaf(c, Vs[jg + 4 * m][bb], acc[m]);
    }
    __syncthreads();
  }
  const int a = a0 + al;
  if (a < d) {
#pragma unroll
    for (int m = 0; m < kPer; ++m) {
      int j = jg + 4 * m;
      if (j < r) Y[((size_t)g * r + j) * d + a] = acc[m];
    }
  }
}

__device__ float block_sum(float v, float* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float s = 0.f;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// One CTA per grain: the r rows of Y (each of length d) made orthonormal by
// modified Gram-Schmidt, each row orthogonalised twice. A row that vanishes
// (a grain with fewer rows than r, or an empty grain) is replaced by a
// coordinate vector and orthogonalised again, which completes the basis.
__global__ void __launch_bounds__(256) k_mgs(const float* Y, int d, int r, float* V) {  // Y may alias V
  extern __shared__ float sv[];  // [r][d]
  __shared__ float red[32];
  const int g = blockIdx.x;
  const float* Yg = Y + (size_t)g * r * d;
  for (int e = threadIdx.x; e < r * d; e += blockDim.x) sv[e] = Yg[e];
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    float* vj = sv + (size_t)j * d;
    float orig = 0.f;
    for (int t = threadIdx.x; t < d; t += blockDim.x) orig += vj[t] * vj[t];
    orig = block_sum(orig, red);
    int fill = 0;
    for (int attempt = 0; attempt <= d; ++attempt) {
      for (int pass = 0; pass < 2; ++pass) {
        for (int i = 0; i < j; ++i) {
          const float* vi = sv + (size_t)i * d;
          float p = 0.f;
          for (int t = threadIdx.x; t < d; t += blockDim.x) p += vi[t] * vj[t];
          p = block_sum(p, red);
          for (int t = threadIdx.x; t < d; t += blockDim.x) vj[t] -= p * vi[t];
          __syncthreads();
        }
      }
      float nn = 0.f;
      for (int t = threadIdx.x; t < d; t += blockDim.x) nn += vj[t] * vj[t];
      nn = block_sum(nn, red);
      if (nn > 1e-10f * fmaxf(orig, 1e-30f) && nn > 1e-30f) {
        const float inv = rsqrtf(nn);
        for (int t = threadIdx.x; t < d; t += blockDim.x) vj[t] *= inv;
        __syncthreads();
        break;
      }
      // degenerate: restart this row from a coordinate vector
      const int c = (j + fill++) % d;
      for (int t = threadIdx.x; t < d; t += blockDim.x) vj[t] = t == c ? 1.f : 0.f;
      orig = 1.f;
      __syncthreads();
    }
  }
  float* Vg = V + (size_t)g * r * d;
  for (int e = threadIdx.x; e < r * d; e += blockDim.x) Vg[e] = sv[e];
}

// ------------------------------------------------------------------ layout

__global__ void k_grain_absmax(const float* __restrict__ Zg, const uint32_t* __restrict__ goff, int r,
                               float* __restrict__ absmax) {
  __shared__ float red[32];
  const int g = blockIdx.x;
  const size_t s = (size_t)goff[g] * r, e = (size_t)goff[g + 1] * r;
  float m = 0.f;
  for (size_t i = s + threadIdx.x; i < e; i += blockDim.x) m = fmaxf(m, fabsf(Zg[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float mm = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) mm = fmaxf(mm, red[i]);
    absmax[g] = mm > 0.f ? mm / 448.f : 1.f;  // FP8 scale s_g
  }
}

// grain-ordered rows -> 128-row Block-SoA blocks (FP32 or FP8 coordinates)
__global__ void k_relayout(int64_t N, int r, int rp, int G, const uint32_t* __restrict__ goff,
                           const uint32_t* __restrict__ blk_off, const uint32_t* __restrict__ ids_g,
                           const float* __restrict__ Zg, const float* __restrict__ rho_g,
                           const int64_t* __restrict__ attr, const float* __restrict__ scale, float* __restrict__ Zb,
                           uint8_t* __restrict__ Z8b, float* __restrict__ rho_b, uint32_t* __restrict__ ids_b,
                           int64_t* __restrict__ attr_b, const uint32_t* __restrict__ slot) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  int lo = 0, hi = G;  // largest g with goff[g] <= p
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (goff[mid] <= (uint32_t)p) lo = mid;
    else hi = mid;
  }
  const int g = lo;
  const uint32_t i = slot[p];  // the row's place within its grain (rows ordered by first coordinate)
  const size_t b = blk_off[g] + i / kBlockRows, t = i % kBlockRows;
  for (int j = 0; j < r; ++j) {
    float z = Zg[(size_t)p * r + j];
    if (Zb) Zb[zoff(b, j, (int)t, rp, 4)] = z;
    if (Z8b)
      Z8b[zoff(b, j, (int)t, rp, 16)] =
          (uint8_t)__nv_cvt_float_to_fp8(z / scale[g], __NV_SATFINITE, __NV_E4M3);
  }
  rho_b[b * kBlockRows + t] = rho_g[p];
  const uint32_t id = ids_g[p];
  ids_b[b * kBlockRows + t] = id;
  if (attr_b) attr_b[b * kBlockRows + t] = attr[id];
}

// smallest residual norm of the real rows of each block (+inf for none)
__global__ void k_block_rho_min(const float* __restrict__ rho_b, const uint32_t* __restrict__ blk_grain,
                                const uint32_t* __restrict__ blk_off, const uint32_t* __restrict__ grain_rows,
                                int64_t nb, float* __restrict__ out) {
  const int64_t b = blockIdx.x;
  if (b >= nb) return;
  const uint32_t g = blk_grain[b];
  const uint32_t row = (uint32_t)(b - blk_off[g]) * kBlockRows + threadIdx.x;
  float v = row < grain_rows[g] ? rho_b[b * kBlockRows + threadIdx.x] : INFINITY;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __shared__ float red[kBlockRows / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = red[0];
    for (int i = 1; i < kBlockRows / 32; ++i) m = fminf(m, red[i]);
    out[b] = m;
  }
}

__global__ void k_to_bf16(const float* __restrict__ X, int64_t n, uint16_t* __restrict__ Xh) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    __nv_bfloat16 h = __float2bfloat16_rn(X[i]);
    Xh[i] = *reinterpret_cast<uint16_t*>(&h);
  }
}

// The second BF16 part of each value, bf16(x - bf16(x)): bf16(x) + it carries
// 16 significant bits of x, exactly (the refined rerank's rows).
__global__ void k_to_bf16_lo(const float* __restrict__ X, int64_t n, uint16_t* __restrict__ Xl) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float x = X[i];
    const float hi = __bfloat162float(__float2bfloat16_rn(x));
    Xl[i] = __bfloat16_as_ushort(__float2bfloat16_rn(x - hi));
  }
}

__global__ void k_fill_u32(uint32_t* p, int64_t n, uint32_t v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// ------------------------------------------------------------------ host

struct Tmp {
  std::vector<void*> ptrs;
  ~Tmp() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  T* get(size_t n, int* rc) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(n * sizeof(T), 16)) != cudaSuccess) {
      *rc = fail(HNTL_ENOMEM, "builder: device allocation of " + std::to_string(n * sizeof(T)) + " bytes failed");
      return nullptr;
    }
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
};

unsigned long long splitmix(unsigned long long& s) {
  unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int nearest(const float* X, int64_t n, const float* M, int G, int d, unsigned long long* packed, cudaStream_t st) {
  HNTL_CUDA_TRY(cudaMemsetAsync(packed, 0xFF, sizeof(unsigned long long) * n, st));
  const int64_t chunk = (int64_t)kNT * 65535;
  for (int64_t s = 0; s < n; s += chunk) {
    int64_t m = std::min(chunk, n - s);
    dim3 grid((G + kNT - 1) / kNT, (unsigned)((m + kNT - 1) / kNT));
    k_nearest<false><<<grid, 256, 0, st>>>(X + s * d, m, M, G, d, packed + s, nullptr);
  }
  HNTL_CUDA_TRY(cudaGetLastError());
  return HNTL_OK;
}

// Capacity-bounded grains (hntl_build_params.max_grain_rows): deferred
// acceptance with rows proposing (Gale and Shapley, 1962). A row proposes to
// the centres in order of (distance, grain); a centre keeps the `cap` rows it
// ranks best by (distance, row) and refuses the rest. The row-proposing stable
// assignment does not depend on the order of the proposals, so the host runs
// the classic loop over ranked lists the GPU prepares (FP32 distances summed
// over t = 0 .. d-1 by fmaf, as the nearest-centre pass forms them): first
// every row's 8 nearest centres; rows refused by all of those wait until the
// proposals stop, then get their 64, 512 and finally all G nearest centres
// in batches and go on proposing from where they stopped. cap * G >= N.
constexpr int kTopK = 8;

// Ranked lists of `m` rows (row ids `rows`, or rows s .. s+m-1 of dX when
// rows is null): the K nearest (distance bits << 32 | grain) keys of each.
int ranked_lists(const float* dX, uint32_t d, uint32_t G, const float* M, const uint32_t* h_rows, int64_t s,
                 int64_t m, int K, unsigned long long* h_out, Tmp& T, float* tile, int64_t R, float* gath,
                 uint64_t* d_rows, unsigned long long* d_top, cudaStream_t st) {
  if (K == kTopK) {  // fused distances and selection, no distance tile (every row's first list)
    for (int64_t c0 = 0; c0 < m; c0 += R) {
      const int64_t mc = std::min<int64_t>(R, m - c0);
      const uint64_t* rows = nullptr;
      if (h_rows) {
        std::vector<uint64_t> rr(mc);
        for (int64_t i = 0; i < mc; ++i) rr[i] = h_rows[c0 + i];
        HNTL_CUDA_TRY(cudaMemcpyAsync(d_rows, rr.data(), mc * 8, cudaMemcpyHostToDevice, st));
        HNTL_CUDA_TRY(cudaStreamSynchronize(st));
        rows = d_rows;
      }
      const float* src = h_rows ? dX : dX + (size_t)(s + c0) * d;
      const unsigned blocks = (unsigned)((mc + kNT - 1) / kNT);
      k_nearest_topk<kTopK><<<blocks, 256, 0, st>>>(src, rows, mc, M, (int)G, (int)d, d_top);
      HNTL_CUDA_TRY(cudaGetLastError());
      HNTL_CUDA_TRY(cudaMemcpyAsync(h_out + (size_t)c0 * K, d_top, (size_t)mc * K * 8, cudaMemcpyDeviceToHost, st));
      HNTL_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return HNTL_OK;
  }
  for (int64_t c0 = 0; c0 < m; c0 += R) {
    const int64_t mc = std::min<int64_t>(R, m - c0);
    const float* src = dX + (size_t)(s + c0) * d;
    if (h_rows) {
      std::vector<uint64_t> rr(mc);
      for (int64_t i = 0; i < mc; ++i) rr[i] = h_rows[c0 + i];
      HNTL_CUDA_TRY(cudaMemcpyAsync(d_rows, rr.data(), mc * 8, cudaMemcpyHostToDevice, st));
      k_gather_rows<<<(unsigned)mc, 256, 0, st>>>(dX, d_rows, mc, (int)d, gath);
      src = gath;
    }
    for (int64_t s2 = 0; s2 < mc; s2 += (int64_t)kNT * 65535) {
      const int64_t m2 = std::min<int64_t>((int64_t)kNT * 65535, mc - s2);
      dim3 grid((G + kNT - 1) / kNT, (unsigned)((m2 + kNT - 1) / kNT));
      k_nearest<true><<<grid, 256, 0, st>>>(src + s2 * d, m2, M, (int)G, (int)d, nullptr, tile + s2 * G);
    }
    k_topk_rows<<<(unsigned)((mc * 32 + 255) / 256), 256, 0, st>>>(tile, mc, (int)G, K, d_top);
    HNTL_CUDA_TRY(cudaGetLastError());
    HNTL_CUDA_TRY(cudaMemcpyAsync(h_out + (size_t)c0 * K, d_top, (size_t)mc * K * 8, cudaMemcpyDeviceToHost, st));
    HNTL_CUDA_TRY(cudaStreamSynchronize(st));
  }
  (void)T;
  return HNTL_OK;
}

int balanced_assign(const float* dX, uint64_t N, uint32_t d, uint32_t G, const float* M, uint32_t cap,
                    int32_t* assign_dev, Tmp& T, cudaStream_t st) {
  int rc = HNTL_OK;
  // row chunks whose G distances fit a 1 GiB tile; a chunk's lists are at most R * G keys
  const int64_t R = std::min<int64_t>((int64_t)N, std::max<int64_t>(kNT, ((int64_t)1 << 28) / (int64_t)G / kNT * kNT));
  float* tile = T.get<float>((size_t)R * G, &rc);
  float* gath = T.get<float>((size_t)R * d, &rc);
  uint64_t* d_rows = T.get<uint64_t>((size_t)R, &rc);
  const int K0 = (int)std::min<uint32_t>(kTopK, G);
  unsigned long long* d_top = T.get<unsigned long long>((size_t)R * G, &rc);
  if (rc) return rc;
  std::vector<unsigned long long> h_top((size_t)N * K0);
  if ((rc = ranked_lists(dX, d, G, M, nullptr, 0, (int64_t)N, K0, h_top.data(), T, tile, R, gath, d_rows, d_top,
                         st)))
    return rc;
  // longer lists of the rows that ran out: list index per row (0 = the first K0)
  std::vector<int32_t> lst(N, -1);
  std::vector<std::vector<unsigned long long>> ext;
  std::vector<int> ext_k;
  // held rows of each centre: a max-heap on (distance bits, row), worst on top
  using Held = std::pair<uint32_t, uint32_t>;
  std::vector<std::vector<Held>> heap(G);
  std::vector<uint32_t> next(N, 0);
  std::vector<int32_t> assign(N, -1);
  std::vector<uint32_t> stack(N), waiting;
  for (uint64_t i = 0; i < N; ++i) stack[i] = (uint32_t)(N - 1 - i);
  for (;;) {
    while (!stack.empty()) {
      const uint32_t i = stack.back();
      stack.pop_back();
      const int k = lst[i] < 0 ? K0 : ext_k[lst[i]];
      if (next[i] >= (uint32_t)k) {  // refused by every listed centre: wait for a longer list
        if (k >= (int)G) return fail(HNTL_ECUDA, "balanced assignment: a row was refused by every centre");
        waiting.push_back(i);
        continue;
      }
      const unsigned long long key =
          lst[i] < 0 ? h_top[(size_t)i * K0 + next[i]] : ext[lst[i]][(size_t)0 + next[i]];
      ++next[i];
      const uint32_t g = (uint32_t)(key & 0xFFFFFFFFu);
      const Held me{(uint32_t)(key >> 32), i};
      auto& h = heap[g];
      if (h.size() < cap) {
        h.push_back(me);
        std::push_heap(h.begin(), h.end());
        assign[i] = (int32_t)g;
      } else if (me < h.front()) {
        std::pop_heap(h.begin(), h.end());
        const uint32_t out = h.back().second;
        h.back() = me;
        std::push_heap(h.begin(), h.end());
        assign[i] = (int32_t)g;
        assign[out] = -1;
        stack.push_back(out);
      } else {
        stack.push_back(i);
      }
    }
    if (waiting.empty()) break;
    // the waiting rows' next lists, in one batch: 64, 512, then every centre
    const int cur = lst[waiting[0]] < 0 ? K0 : ext_k[lst[waiting[0]]];
    int K = cur < 64 ? 64 : (cur < 512 ? 512 : (int)G);
    K = std::min<int>(K, (int)G);
    for (uint32_t i : waiting) {  // rows of different list lengths: the longest one decides
      const int ki = lst[i] < 0 ? K0 : ext_k[lst[i]];
      if (ki >= K) K = std::min<int>((int)G, ki < 512 ? 512 : (int)G);
    }
    std::vector<unsigned long long> h_ext(waiting.size() * (size_t)K);
    const int64_t Rk = std::max<int64_t>(1, std::min<int64_t>(R, ((int64_t)R * G) / K));
    if ((rc = ranked_lists(dX, d, G, M, waiting.data(), 0, (int64_t)waiting.size(), K, h_ext.data(), T, tile,
                           std::min<int64_t>(R, Rk), gath, d_rows, d_top, st)))
      return rc;
    for (size_t w = 0; w < waiting.size(); ++w) {
      ext.emplace_back(h_ext.begin() + w * K, h_ext.begin() + (w + 1) * K);
      ext_k.push_back(K);
      lst[waiting[w]] = (int32_t)(ext.size() - 1);
      stack.push_back(waiting[w]);
    }
    waiting.clear();
  }
  HNTL_CUDA_TRY(cudaMemcpyAsync(assign_dev, assign.data(), N * 4, cudaMemcpyHostToDevice, st));
  HNTL_CUDA_TRY(cudaStreamSynchronize(st));
  return HNTL_OK;
}

template <int RT>
void cov_apply(const float* C, const float* V, int d, int r, int gb, float* Y, cudaStream_t st) {
  dim3 grid((d + kCT - 1) / kCT, gb);
  k_cov_apply<RT><<<grid, 256, 0, st>>>(C, V, d, r, Y);
}

}  // namespace

int build_index(const float* dX, uint64_t N, uint32_t d, uint32_t G, uint32_t r, const hntl_build_params* prm,
                int device, cudaStream_t st, Index& I) {
  if (!dX || N == 0 || d == 0 || G == 0 || r == 0 || r > d) return fail(HNTL_EINVAL, "bad builder sizes");
  if (r > (uint32_t)kMaxR) return fail(HNTL_EINVAL, "r > 64 is not supported");
  if (G > kMaxG) return fail(HNTL_EINVAL, "more than 8192 grains is not supported");
  if (N < G) return fail(HNTL_EINVAL, "fewer rows than grains");
  if (N >= (1ull << 32) - 1) return fail(HNTL_EINVAL, "too many rows");
  hntl_build_params P{};
  if (prm) P = *prm;
  const bool rprune = P.precision & HNTL_INT16_RESID_PRUNE;
  const bool refine = P.precision & HNTL_RERANK_REFINE;
  const uint32_t precision = P.precision & ~(HNTL_INT16_RESID_PRUNE | HNTL_RERANK_REFINE);
  if (precision != HNTL_PREC_FP32 && precision != HNTL_PREC_BF16_FP8 && precision != HNTL_PREC_INT16)
    return fail(HNTL_EINVAL, "bad precision");
  if (rprune && precision != HNTL_PREC_INT16)
    return fail(HNTL_EINVAL, "residual-saturation pruning applies to the 16-bit form only");
  if (refine && precision != HNTL_PREC_BF16_FP8)
    return fail(HNTL_EINVAL, "the refined rerank applies to the precision form only");
  if (precision == HNTL_PREC_BF16_FP8 && d % 8)  // BF16 rows move in 16-byte pieces
    return fail(HNTL_EINVAL, "the precision form needs d to be a multiple of 8");
  const uint32_t max_iter = P.max_iter ? P.max_iter : 10;
  const uint32_t pca_iters = P.pca_iters ? P.pca_iters : 12;
  const uint64_t n_t = std::min<uint64_t>(N, P.n_train ? P.n_train : 256ull * G);
  const uint64_t n_s = std::min<uint64_t>(n_t, P.n_seed ? P.n_seed : 32ull * G);
  if (n_s < G) return fail(HNTL_EINVAL, "seeding subset smaller than G");
  if (P.max_grain_rows && (uint64_t)P.max_grain_rows * G < N)
    return fail(HNTL_EINVAL, "max_grain_rows * G must be at least N");
  std::vector<double> u(G);
  if (P.u) {
    std::memcpy(u.data(), P.u, sizeof(double) * G);
  } else {
    unsigned long long s = P.seed ^ 0x5EEDull;
    for (uint32_t g = 0; g < G; ++g) u[g] = (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
  }
  for (double x : u)
    if (!(x >= 0.0 && x < 1.0)) return fail(HNTL_EINVAL, "k-means++ draws must lie in [0, 1)");

  int rc = HNTL_OK;
  Tmp T;
  // --- training and seeding subsets (strided rows)
  std::vector<uint64_t> h_rows(n_t);
  for (uint64_t i = 0; i < n_t; ++i) h_rows[i] = (i * N) / n_t;
  std::vector<uint64_t> h_srows(n_s);
  for (uint64_t i = 0; i < n_s; ++i) h_srows[i] = (i * n_t) / n_s;
  uint64_t* d_rows = T.get<uint64_t>(n_t, &rc);
  uint64_t* d_srows = T.get<uint64_t>(n_s, &rc);
  float* Xt = T.get<float>(n_t * d, &rc);
  float* Xs = T.get<float>(n_s * d, &rc);
  float* M = nullptr;
  float* dmin = T.get<float>(n_s, &rc);
  long long* d_chosen = T.get<long long>(G, &rc);
  if (rc) return rc;
  HNTL_CUDA_TRY(cudaMemcpyAsync(d_rows, h_rows.data(), n_t * 8, cudaMemcpyHostToDevice, st));
  HNTL_CUDA_TRY(cudaMemcpyAsync(d_srows, h_srows.data(), n_s * 8, cudaMemcpyHostToDevice, st));
  k_gather_rows<<<(unsigned)n_t, 256, 0, st>>>(dX, d_rows, (int64_t)n_t, (int)d, Xt);
  k_gather_rows<<<(unsigned)n_s, 256, 0, st>>>(Xt, d_srows, (int64_t)n_s, (int)d, Xs);

  // index-owned arrays
  I = Index();
  I.device = device;
  I.n = N;
  I.d = d;
  I.G = G;
  I.r = r;
  I.precision = precision;
  I.i16_resid_prune = rprune;
  I.rp = (uint32_t)padded_r((int)r, (int)precision);
  I.has_attr = P.d_attr != nullptr;
  auto own = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
    I.allocations.push_back(p);
    I.device_bytes += std::max<size_t>(bytes, 16);
    return p;
  };
  auto cleanup = [&]() {
    for (void* p : I.allocations) cudaFree(p);
    I.allocations.clear();
  };
  M = static_cast<float*>(own((size_t)G * d * 4));
  I.U = static_cast<float*>(own((size_t)G * r * d * 4));
  if (!M || !I.U) {
    cleanup();
    return fail(HNTL_ENOMEM, "builder: index allocation failed");
  }
  I.M = M;

  // --- k-means++ seeding on Xs
  {
    long long first = (long long)(u[0] * (double)n_s);
    if (first >= (long long)n_s) first = (long long)n_s - 1;
    HNTL_CUDA_TRY(cudaMemcpyAsync(M, Xs + (size_t)first * d, (size_t)d * 4, cudaMemcpyDeviceToDevice, st));
    const unsigned wb = (unsigned)((n_s * 32 + 255) / 256);
    k_kpp_dist<<<wb, 256, 0, st>>>(Xs, (int64_t)n_s, (int)d, M, dmin, 1);
    for (uint32_t c = 1; c < G; ++c) {
      k_kpp_pick<<<1, 1024, 0, st>>>(dmin, (int64_t)n_s, u[c], Xs, (int)d, M + (size_t)c * d, d_chosen + c);
      k_kpp_dist<<<wb, 256, 0, st>>>(Xs, (int64_t)n_s, (int)d, M + (size_t)c * d, dmin, 0);
    }
    HNTL_CUDA_TRY(cudaGetLastError());
  }

  // --- Lloyd iterations on Xt
  unsigned long long* packed = T.get<unsigned long long>(std::max<uint64_t>(n_t, N), &rc);
  int32_t* assign = T.get<int32_t>(std::max<uint64_t>(n_t, N), &rc);
  int32_t* prev = T.get<int32_t>(n_t, &rc);
  float* dist = T.get<float>(n_t, &rc);
  double* sums = T.get<double>((size_t)G * d, &rc);
  unsigned int* counts = T.get<unsigned int>(G, &rc);
  unsigned int* changed = T.get<unsigned int>(1, &rc);
  if (rc) {
    cleanup();
    return rc;
  }
  HNTL_CUDA_TRY(cudaMemsetAsync(prev, 0xFF, n_t * 4, st));
  std::vector<unsigned int> h_counts(G);
  for (uint32_t it = 0; it < max_iter; ++it) {
    if ((rc = nearest(Xt, (int64_t)n_t, M, (int)G, (int)d, packed, st))) break;
    HNTL_CUDA_TRY(cudaMemsetAsync(changed, 0, 4, st));
    k_unpack<<<(unsigned)((n_t + 255) / 256), 256, 0, st>>>(packed, (int64_t)n_t, assign, dist, prev, changed);
    unsigned int h_changed = 0;
    HNTL_CUDA_TRY(cudaMemcpyAsync(&h_changed, changed, 4, cudaMemcpyDeviceToHost, st));
    HNTL_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_changed == 0) break;
    HNTL_CUDA_TRY(cudaMemcpyAsync(prev, assign, n_t * 4, cudaMemcpyDeviceToDevice, st));
    HNTL_CUDA_TRY(cudaMemsetAsync(sums, 0, (size_t)G * d * 8, st));
    HNTL_CUDA_TRY(cudaMemsetAsync(counts, 0, (size_t)G * 4, st));
    k_accum<<<(unsigned)((n_t * 32 + 255) / 256), 256, 0, st>>>(Xt, (int64_t)n_t, (int)d, assign, sums, counts);
    k_means_finalize<<<(unsigned)(((size_t)G * d + 255) / 256), 256, 0, st>>>(sums, counts, (int)G, (int)d, M);
    HNTL_CUDA_TRY(cudaMemcpyAsync(h_counts.data(), counts, (size_t)G * 4, cudaMemcpyDeviceToHost, st));
    HNTL_CUDA_TRY(cudaStreamSynchronize(st));
    // empty grains take the training rows farthest from their own centre
    std::vector<uint32_t> empty;
    for (uint32_t g = 0; g < G; ++g)
      if (!h_counts[g]) empty.push_back(g);
    if (!empty.empty()) {
      std::vector<float> h_dist(n_t);
      HNTL_CUDA_TRY(cudaMemcpy(h_dist.data(), dist, n_t * 4, cudaMemcpyDeviceToHost));
      std::vector<uint64_t> order(n_t);
      for (uint64_t i = 0; i < n_t; ++i) order[i] = i;
      std::stable_sort(order.begin(), order.end(), [&](uint64_t a, uint64_t b) { return h_dist[a] > h_dist[b]; });
      for (size_t e = 0; e < empty.size() && e < n_t; ++e)
        HNTL_CUDA_TRY(cudaMemcpyAsync(M + (size_t)empty[e] * d, Xt + order[e] * d, (size_t)d * 4,
                                      cudaMemcpyDeviceToDevice, st));
    }
  }
  if (rc) {
    cleanup();
    return rc;
  }

  // --- final assignment of all rows (nearest centre, or capacity-bounded), exact means of final members
  if (P.max_grain_rows) {
    if ((rc = balanced_assign(dX, N, d, G, M, P.max_grain_rows, assign, T, st))) {
      cleanup();
      return rc;
    }
  } else {
    if ((rc = nearest(dX, (int64_t)N, M, (int)G, (int)d, packed, st))) {
      cleanup();
      return rc;
    }
    k_unpack<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(packed, (int64_t)N, assign, nullptr, nullptr, nullptr);
  }
  HNTL_CUDA_TRY(cudaMemsetAsync(sums, 0, (size_t)G * d * 8, st));
  HNTL_CUDA_TRY(cudaMemsetAsync(counts, 0, (size_t)G * 4, st));
  k_accum<<<(unsigned)((N * 32 + 255) / 256), 256, 0, st>>>(dX, (int64_t)N, (int)d, assign, sums, counts);
  k_means_finalize<<<(unsigned)(((size_t)G * d + 255) / 256), 256, 0, st>>>(sums, counts, (int)G, (int)d, M);

  // grain order on the host: stable counting sort of ids by grain
  std::vector<int32_t> h_assign(N);
  HNTL_CUDA_TRY(cudaMemcpyAsync(h_assign.data(), assign, N * 4, cudaMemcpyDeviceToHost, st));
  HNTL_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<uint32_t> h_goff(G + 1, 0), h_ids(N);
  for (uint64_t i = 0; i < N; ++i) h_goff[h_assign[i] + 1]++;
  for (uint32_t g = 0; g < G; ++g) h_goff[g + 1] += h_goff[g];
  {
    std::vector<uint32_t> cur(h_goff.begin(), h_goff.end() - 1);
    for (uint64_t i = 0; i < N; ++i) h_ids[cur[h_assign[i]]++] = (uint32_t)i;
  }
  uint32_t* goff = T.get<uint32_t>(G + 1, &rc);
  uint32_t* ids_g = T.get<uint32_t>(N, &rc);
  if (rc) {
    cleanup();
    return rc;
  }
  HNTL_CUDA_TRY(cudaMemcpyAsync(goff, h_goff.data(), (G + 1) * 4, cudaMemcpyHostToDevice, st));
  HNTL_CUDA_TRY(cudaMemcpyAsync(ids_g, h_ids.data(), N * 4, cudaMemcpyHostToDevice, st));

  // --- local bases by orthogonal iteration on the grain covariances (batches of grains)
  {
    const size_t dd = (size_t)d * d;
    const size_t budget = (size_t)8 << 30;
    const uint32_t gb = (uint32_t)std::max<size_t>(1, std::min<size_t>(G, budget / (dd * 4)));
    float* C = T.get<float>(gb * dd, &rc);
    float* Y = T.get<float>((size_t)gb * r * d, &rc);
    if (rc) {
      cleanup();
      return rc;
    }
    const int nt = (d + kCT - 1) / kCT;
    const size_t smem = (size_t)r * d * 4;
    if (smem > 227 * 1024) {
      cleanup();
      return fail(HNTL_EINVAL, "builder: r * d too large for the in-shared-memory Gram-Schmidt");
    }
    HNTL_CUDA_TRY(cudaFuncSetAttribute(k_mgs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_init_basis<<<(unsigned)(((size_t)G * r * d + 255) / 256), 256, 0, st>>>(I.U, (int64_t)G * r * d,
                                                                               P.seed + 0xB45Eull);
    for (uint32_t g0 = 0; g0 < G; g0 += gb) {
      const uint32_t nb = std::min(gb, G - g0);
      float* Ub = I.U + (size_t)g0 * r * d;
      k_cov<<<dim3(nt * (nt + 1) / 2, nb), 256, 0, st>>>(dX, ids_g, goff, M, (int)d, (int)g0, C);
      k_mgs<<<nb, 256, smem, st>>>(Ub, (int)d, (int)r, Ub);
      for (uint32_t it = 0; it < pca_iters; ++it) {
        if (r <= 8) cov_apply<8>(C, Ub, (int)d, (int)r, (int)nb, Y, st);
        else if (r <= 16) cov_apply<16>(C, Ub, (int)d, (int)r, (int)nb, Y, st);
        else if (r <= 32) cov_apply<32>(C, Ub, (int)d, (int)r, (int)nb, Y, st);
        else cov_apply<64>(C, Ub, (int)d, (int)r, (int)nb, Y, st);
        k_mgs<<<nb, 256, smem, st>>>(Y, (int)d, (int)r, Ub);
      }
    }
    HNTL_CUDA_TRY(cudaGetLastError());
  }

  // --- database coordinates and residual norms (Eq. 1-4), grain order
  float* Zg = T.get<float>((size_t)N * r, &rc);
  float* rho_g = T.get<float>(N, &rc);
  uint32_t* grp_off = T.get<uint32_t>(G + 1, &rc);
  if (rc) {
    cleanup();
    return rc;
  }
  {
    std::vector<uint32_t> h_grp(G + 1, 0);
    for (uint32_t g = 0; g < G; ++g)
      h_grp[g + 1] = h_grp[g] + (h_goff[g + 1] - h_goff[g] + kPairsPerGroup - 1) / kPairsPerGroup;
    HNTL_CUDA_TRY(cudaMemcpyAsync(grp_off, h_grp.data(), (G + 1) * 4, cudaMemcpyHostToDevice, st));
    size_t smem = (size_t)kPairsPerGroup * d * sizeof(float);
    if (smem > 40 * 1024)  // the kernel's static shared memory counts against the default 48 KB too
      HNTL_CUDA_TRY(cudaFuncSetAttribute(k_project<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    unsigned grid = (unsigned)std::min<uint64_t>(h_grp[G] ? h_grp[G] : 1, 148 * 32);
    k_project<false><<<grid, 256, smem, st>>>(dX, M, I.U, (int)d, (int)r, (int)G, grp_off, goff, ids_g, Zg, rho_g);
    HNTL_CUDA_TRY(cudaGetLastError());
  }

  // --- Block-SoA layout
  I.h_blk_off.assign(G + 1, 0);
  std::vector<uint32_t> h_rows_g(G), h_blk_grain;
  std::vector<uint64_t> padded(G);
  for (uint32_t g = 0; g < G; ++g) {
    uint32_t ng = h_goff[g + 1] - h_goff[g];
    h_rows_g[g] = ng;
    uint32_t nbk = (ng + kBlockRows - 1) / kBlockRows;
    I.h_blk_off[g + 1] = I.h_blk_off[g] + nbk;
    padded[g] = (uint64_t)nbk * kBlockRows;
    I.max_grain_rows = std::max<uint64_t>(I.max_grain_rows, ng);
    for (uint32_t b = 0; b < nbk; ++b) h_blk_grain.push_back(g);
  }
  I.n_blocks = I.h_blk_off[G];
  {
    std::vector<uint64_t> sorted = padded;
    std::sort(sorted.begin(), sorted.end(), std::greater<uint64_t>());
    I.h_top_padded_prefix.assign(G + 1, 0);
    for (uint32_t g = 0; g < G; ++g) I.h_top_padded_prefix[g + 1] = I.h_top_padded_prefix[g] + sorted[g];
  }
  const size_t rows_pad = I.n_blocks * kBlockRows;
  I.blk_off = static_cast<uint32_t*>(own((G + 1) * 4));
  I.grain_rows = static_cast<uint32_t*>(own(G * 4));
  I.blk_grain = static_cast<uint32_t*>(own(I.n_blocks * 4));
  I.rho = static_cast<float*>(own(rows_pad * 4));
  I.blk_rho_min = static_cast<float*>(own(I.n_blocks * 4));
  I.ids = static_cast<uint32_t*>(own(rows_pad * 4));
  if (I.has_attr) I.attr_b = static_cast<int64_t*>(own(rows_pad * 8));
  if (precision == HNTL_PREC_FP32 || precision == HNTL_PREC_INT16) {  // the 16-bit form is derived below
    I.Zb = static_cast<float*>(own(rows_pad * I.rp * 4));
    I.X = static_cast<float*>(own(N * d * 4));
  } else {
    I.Z8b = static_cast<uint8_t*>(own(rows_pad * I.rp));
    I.scale = static_cast<float*>(own(G * 4));
    I.Xh = static_cast<uint16_t*>(own(N * d * 2));
    if (refine) I.Xl = static_cast<uint16_t*>(own(N * d * 2));
  }
  if (!I.blk_off || !I.grain_rows || !I.blk_grain || !I.rho || !I.blk_rho_min || !I.ids || (I.has_attr && !I.attr_b) ||
      (precision != HNTL_PREC_BF16_FP8 ? (!I.Zb || !I.X) : (!I.Z8b || !I.scale || !I.Xh || (refine && !I.Xl)))) {
    cleanup();
    return fail(HNTL_ENOMEM, "builder: index allocation failed");
  }
  HNTL_CUDA_TRY(cudaMemcpyAsync(I.blk_off, I.h_blk_off.data(), (G + 1) * 4, cudaMemcpyHostToDevice, st));
  HNTL_CUDA_TRY(cudaMemcpyAsync(I.grain_rows, h_rows_g.data(), G * 4, cudaMemcpyHostToDevice, st));
  HNTL_CUDA_TRY(cudaMemcpyAsync(I.blk_grain, h_blk_grain.data(), I.n_blocks * 4, cudaMemcpyHostToDevice, st));
  HNTL_CUDA_TRY(cudaMemsetAsync(I.rho, 0, rows_pad * 4, st));
  k_fill_u32<<<(unsigned)((rows_pad + 255) / 256), 256, 0, st>>>(I.ids, (int64_t)rows_pad, kInvalidId);
  if (I.attr_b) HNTL_CUDA_TRY(cudaMemsetAsync(I.attr_b, 0, rows_pad * 8, st));
  if (I.Zb) HNTL_CUDA_TRY(cudaMemsetAsync(I.Zb, 0, rows_pad * I.rp * 4, st));
  if (I.Z8b) {
    HNTL_CUDA_TRY(cudaMemsetAsync(I.Z8b, 0, rows_pad * I.rp, st));
    k_grain_absmax<<<G, 256, 0, st>>>(Zg, goff, (int)r, I.scale);
  }
  // within a grain, rows go to blocks in order of their first coordinate (the scan's interval bound)
  std::vector<uint64_t> order;
  {
    std::vector<float> z0(N);
    HNTL_CUDA_TRY(cudaStreamSynchronize(st));
    HNTL_CUDA_TRY(cudaMemcpy2D(z0.data(), 4, Zg, (size_t)r * 4, 4, N, cudaMemcpyDeviceToHost));
    std::vector<uint64_t> go(G + 1);
    for (uint32_t g = 0; g <= G; ++g) go[g] = h_goff[g];
    order = rows_by_first_coord(z0.data(), 1, h_ids.data(), go);
    std::vector<uint32_t> h_slot(N);
    for (uint32_t g = 0; g < G; ++g)
      for (uint64_t i = go[g]; i < go[g + 1]; ++i) h_slot[order[i]] = (uint32_t)(i - go[g]);
    uint32_t* slot = T.get<uint32_t>(N, &rc);
    if (rc) {
      cleanup();
      return rc;
    }
    HNTL_CUDA_TRY(cudaMemcpy(slot, h_slot.data(), N * 4, cudaMemcpyHostToDevice));
    k_relayout<<<(unsigned)((N + 255) / 256), 256, 0, st>>>((int64_t)N, (int)r, (int)I.rp, (int)G, goff, I.blk_off,
                                                            ids_g, Zg, rho_g, P.d_attr, I.scale, I.Zb, I.Z8b, I.rho,
                                                            I.ids, I.attr_b, slot);
  }
  if (I.n_blocks)
    k_block_rho_min<<<(unsigned)I.n_blocks, kBlockRows, 0, st>>>(I.rho, I.blk_grain, I.blk_off, I.grain_rows,
                                                                 (int64_t)I.n_blocks, I.blk_rho_min);
  if (I.X) HNTL_CUDA_TRY(cudaMemcpyAsync(I.X, dX, N * d * 4, cudaMemcpyDeviceToDevice, st));
  if (I.Xh) k_to_bf16<<<(unsigned)((N * d + 255) / 256), 256, 0, st>>>(dX, (int64_t)(N * d), I.Xh);
  if (I.Xl) k_to_bf16_lo<<<(unsigned)((N * d + 255) / 256), 256, 0, st>>>(dX, (int64_t)(N * d), I.Xl);
  HNTL_CUDA_TRY(cudaGetLastError());
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cleanup();
    return fail(HNTL_ECUDA, std::string("builder: ") + cudaGetErrorString(e));
  }
  if (precision == HNTL_PREC_INT16) {
    // the 16-bit form from the FP32 coordinates, by the loader's own quantiser
    std::vector<float> hz((size_t)N * r), hrho(N);
    HNTL_CUDA_TRY(cudaMemcpy(hz.data(), Zg, hz.size() * 4, cudaMemcpyDeviceToHost));
    HNTL_CUDA_TRY(cudaMemcpy(hrho.data(), rho_g, N * 4, cudaMemcpyDeviceToHost));
    std::vector<uint64_t> go(G + 1);
    for (uint32_t g = 0; g <= G; ++g) go[g] = h_goff[g];
    std::vector<float> delta, dres, rho16;
    std::vector<int16_t> codes;
    int16_quantize(hz.data(), hrho.data(), go, r, delta, dres, codes, rho16);
    const int rp = (int)I.rp;
    std::vector<int16_t> z16(rows_pad * rp, 0);
    std::vector<float> rho_b(rows_pad, 0.0f);
    for (uint32_t g = 0; g < G; ++g)
      for (uint64_t i = 0; i < go[g + 1] - go[g]; ++i) {
        const uint64_t p = order[go[g] + i], b = I.h_blk_off[g] + i / kBlockRows, t = i % kBlockRows;
        for (uint32_t j = 0; j < r; ++j) z16[zoff(b, (int)j, (int)t, rp, 8)] = codes[p * r + j];
        rho_b[b * kBlockRows + t] = rho16[p];
      }
    I.Z16b = static_cast<int16_t*>(own(rows_pad * rp * 2));
    I.scale = static_cast<float*>(own(G * 4));
    I.dres = static_cast<float*>(own(G * 4));
    if (!I.Z16b || !I.scale || !I.dres) {
      cleanup();
      return fail(HNTL_ENOMEM, "builder: 16-bit form allocation failed");
    }
    HNTL_CUDA_TRY(cudaMemcpy(I.Z16b, z16.data(), z16.size() * 2, cudaMemcpyHostToDevice));
    HNTL_CUDA_TRY(cudaMemcpy(I.scale, delta.data(), G * 4, cudaMemcpyHostToDevice));
    HNTL_CUDA_TRY(cudaMemcpy(I.dres, dres.data(), G * 4, cudaMemcpyHostToDevice));
    HNTL_CUDA_TRY(cudaMemcpy(I.rho, rho_b.data(), rows_pad * 4, cudaMemcpyHostToDevice));
    if (I.n_blocks)
      k_block_rho_min<<<(unsigned)I.n_blocks, kBlockRows, 0, st>>>(I.rho, I.blk_grain, I.blk_off, I.grain_rows,
                                                                   (int64_t)I.n_blocks, I.blk_rho_min);
    I.Zb = nullptr;  // the scan reads the 16-bit codes (the FP32 array stays with the index's allocations)
    HNTL_CUDA_TRY(cudaGetLastError());
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cleanup();
      return fail(HNTL_ECUDA, std::string("builder: ") + cudaGetErrorString(e));
    }
  }
  return finalize_index(I);
}

}  // namespace hntl

extern "C" int hntl_index_build(const float* d_X, uint64_t N, uint32_t d, uint32_t G, uint32_t r,
                                const hntl_build_params* params, int device, void* stream, hntl_index** out) {
  hntl::clear_error();
  if (!out) return hntl::fail(HNTL_EINVAL, "null argument");
  *out = nullptr;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return hntl::fail(HNTL_ECUDA, "cannot select the device");
  hntl_index* h = new (std::nothrow) hntl_index();
  if (!h) return hntl::fail(HNTL_ENOMEM, "host allocation failed");
  int rc = hntl::build_index(d_X, N, d, G, r, params, device, static_cast<cudaStream_t>(stream), h->I);
  if (rc != HNTL_OK) hntl::release(h->I);
  if (prev >= 0) cudaSetDevice(prev);
  if (rc != HNTL_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return HNTL_OK;
}
