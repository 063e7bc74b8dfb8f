// Mode B batched search: routing, bucketing, projection, Block-SoA scan,
// pool selection and exact rerank.
//
//   step                      paper                              kernel(s)
//   routing                   sec. 2.1 step 1, sec. 2.3 item 1   k_route_dist, k_route_select
//   (query, grain) bucketing  batched form of sec. 2.3 item 2    k_bucket_count/scan/scatter
//   projection                Eq. 1-4                            k_project
//   scan                      Eq. 6, sec. 2.1 step 3, sec. 2.4   k_scan_fp32
//   pool of C                 Table 1 "Pool C"                   k_select
//   exact rerank to k         sec. 2.1 step 4 (Mode B)           k_rerank
//
// Every distance is formed in direct difference form in FP32, the way the
// method states it: routing sum (q_t - mu_t)^2; projection of the centred
// query v' = q - mu_g; residual e = v' - U^T z and rho_q = ||e||^2; scan
// ||z_q - z_i||^2 + rho_q + rho_i; rerank sum (q_t - x_t)^2.
#include <array>
#include <cfloat>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "hntl_internal.cuh"
#include "kernels_common.cuh"
#include "route_kernels.cuh"

namespace hntl {

namespace {

constexpr int kSelThreads = 512;
constexpr int kTieCap = 1024;

__device__ __forceinline__ uint32_t fkey(float x) { return __float_as_uint(x); }  // x >= 0: monotone

// ------------------------------------------------------------------ bucketing

__global__ void k_bucket_count(const int32_t* __restrict__ probe, int n, uint32_t* __restrict__ gcnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&gcnt[probe[i]], 1u);
}

// Single CTA: exclusive scans over grains of the pair counts (pair offsets),
// of count x padded rows (distance-buffer bases) and of projection groups.
__global__ void __launch_bounds__(1024) k_bucket_scan(const uint32_t* __restrict__ gcnt,
                                                      const uint32_t* __restrict__ blk_off, int G,
                                                      uint32_t* __restrict__ pair_off, uint64_t* __restrict__ seg_base,
                                                      uint32_t* __restrict__ grp_off) {
  __shared__ uint32_t ws32[32];
  __shared__ unsigned long long ws64[32];
  __shared__ uint32_t tot32a, tot32b;
  __shared__ unsigned long long tot64;
  uint32_t carry_p = 0, carry_gr = 0;
  unsigned long long carry_s = 0;
  for (int c0 = 0; c0 < G; c0 += 1024) {
    int g = c0 + threadIdx.x;
    uint32_t cnt = g < G ? gcnt[g] : 0u;
    uint32_t pad = g < G ? (blk_off[g + 1] - blk_off[g]) * (uint32_t)kBlockRows : 0u;
    uint32_t ngr = (cnt + kPairsPerGroup - 1) / kPairsPerGroup;
    uint32_t ep = block_exclusive_scan<uint32_t>(cnt, &tot32a, ws32);
    uint32_t eg = block_exclusive_scan<uint32_t>(ngr, &tot32b, ws32);
    unsigned long long es =
        block_exclusive_scan<unsigned long long>((unsigned long long)cnt * pad, &tot64, ws64);
    if (g < G) {
      pair_off[g] = carry_p + ep;
      grp_off[g] = carry_gr + eg;
      seg_base[g] = carry_s + es;
    }
    carry_p += tot32a;
    carry_gr += tot32b;
    carry_s += tot64;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pair_off[G] = carry_p;
    grp_off[G] = carry_gr;
  }
}

__global__ void k_bucket_scatter(const int32_t* __restrict__ probe, int nq, int nprobe,
                                 const uint32_t* __restrict__ pair_off, uint32_t* __restrict__ gcur,
                                 uint32_t* __restrict__ pair_q, uint32_t* __restrict__ pair_of) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq * nprobe) return;
  int g = probe[i];
  uint32_t pos = pair_off[g] + atomicAdd(&gcur[g], 1u);
  pair_q[pos] = (uint32_t)(i / nprobe);
  pair_of[i] = pos;
}

// ------------------------------------------------------------------ scan

// One CTA per Block-SoA block (128 rows, one thread per row). The row's r
// coordinates stay in registers; every (query, grain) pair of the block's
// grain is applied in turn: D = ||z_q - z_i||^2 + rho_q + rho_i (Eq. 6).
// Rows failing the pair's attribute range, and padding rows, get D = +inf.
// D goes to the pair's segment of the distance buffer (row order).
template <int RT>
__global__ void __launch_bounds__(kBlockRows) k_scan_fp32(
    const uint32_t* __restrict__ blk_grain, const uint32_t* __restrict__ blk_off,
    const uint32_t* __restrict__ grain_rows, const float* __restrict__ Zb, const float* __restrict__ rho,
    const int64_t* __restrict__ attr_b, int r, const uint32_t* __restrict__ gcnt,
    const uint32_t* __restrict__ pair_off, const uint64_t* __restrict__ seg_base,
    const uint32_t* __restrict__ pair_q, const float* __restrict__ zq, const float* __restrict__ rhoq,
    const int64_t* __restrict__ filter, float* __restrict__ D) {
  constexpr int kChunk = 32;
  __shared__ float sz[kChunk][RT + 1];
  __shared__ float srho[kChunk];
  __shared__ long long slo[kChunk], shi[kChunk];
  const size_t b = blockIdx.x;
  const uint32_t g = blk_grain[b];
  const uint32_t m = gcnt[g];
  if (m == 0) return;
  const int t = threadIdx.x;
  const uint32_t jb = (uint32_t)b - blk_off[g];
  const uint32_t row = jb * kBlockRows + t;
  const bool valid = row < grain_rows[g];
  const size_t padded = (size_t)(blk_off[g + 1] - blk_off[g]) * kBlockRows;
  float z[RT];
#pragma unroll
  for (int j = 0; j < RT; ++j) z[j] = j < r ? Zb[(b * r + j) * kBlockRows + t] : 0.f;
  const float rho_i = rho[b * kBlockRows + t];
  const long long a = filter ? (long long)attr_b[b * kBlockRows + t] : 0;
  const uint32_t p_begin = pair_off[g];
  float* Dg = D + seg_base[g] + row;
  for (uint32_t s0 = 0; s0 < m; s0 += kChunk) {
    const int ns = (int)min((uint32_t)kChunk, m - s0);
    for (int e = t; e < kChunk * RT; e += kBlockRows) {
      int s = e / RT, j = e - s * RT;
      sz[s][j] = (s < ns && j < r) ? zq[(size_t)(p_begin + s0 + s) * r + j] : 0.f;
    }
    if (t < kChunk) {
      srho[t] = t < ns ? rhoq[p_begin + s0 + t] : 0.f;
      if (filter && t < ns) {
        uint32_t q = pair_q[p_begin + s0 + t];
        slo[t] = (long long)filter[2 * (size_t)q];
        shi[t] = (long long)filter[2 * (size_t)q + 1];
      }
    }
    __syncthreads();
    for (int s = 0; s < ns; ++s) {
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < RT; ++j) {
        float df = sz[s][j] - z[j];
        acc = fmaf(df, df, acc);
      }
      float Dv = acc + srho[s] + rho_i;
      bool ok = valid && (!filter || (a >= slo[s] && a <= shi[s]));
      Dg[(size_t)(s0 + s) * padded] = ok ? Dv : INFINITY;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ pool selection

struct SegIter {
  const float* base;
  uint32_t len;
  uint32_t row0;  // first padded row of the grain
};

__device__ __forceinline__ SegIter seg_of(int q, int p, int nprobe, const int32_t* probe, const uint32_t* pair_of,
                                          const uint32_t* pair_off, const uint64_t* seg_base,
                                          const uint32_t* blk_off, const float* D) {
  const int g = probe[(size_t)q * nprobe + p];
  const uint32_t s = pair_of[(size_t)q * nprobe + p];
  const uint32_t padded = (blk_off[g + 1] - blk_off[g]) * (uint32_t)kBlockRows;
  SegIter it;
  it.base = D + seg_base[g] + (size_t)(s - pair_off[g]) * padded;
  it.len = padded;
  it.row0 = blk_off[g] * (uint32_t)kBlockRows;
  return it;
}

// Bitonic sort of n (a power of two, <= 1024) 64-bit keys in shared memory.
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

// Find the bin holding the need-th smallest (1-based) key of a 2048-bin
// histogram; returns the bin and the count below it.
__device__ void find_bin(const uint32_t* hist, int nbins, uint32_t need, uint32_t* s_bin, uint32_t* s_below,
                         uint32_t* scratch) {
  // each thread sums a contiguous range of bins, exclusive scan, then the owner thread walks its range
  const int per = (nbins + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per;
  uint32_t sum = 0;
  for (int i = 0; i < per; ++i)
    if (b0 + i < nbins) sum += hist[b0 + i];
  uint32_t tot;
  uint32_t* tot_p = scratch + 64;
  uint32_t excl = block_exclusive_scan<uint32_t>(sum, tot_p, scratch);
  (void)tot;
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

// One CTA per query: the exact C smallest (D, id) over the query's probed
// segments, by a three-digit (11/11/10-bit) radix select on the FP32 bit
// pattern of D (non-negative, so bit order is value order), then ties at the
// threshold resolved by id, then a bitonic sort of the C winners.
__global__ void __launch_bounds__(kSelThreads) k_select(
    int nprobe, int C, const int32_t* __restrict__ probe, const uint32_t* __restrict__ pair_of,
    const uint32_t* __restrict__ pair_off, const uint64_t* __restrict__ seg_base, const uint32_t* __restrict__ blk_off,
    const uint32_t* __restrict__ ids, const float* __restrict__ D, uint32_t* __restrict__ cand_id,
    float* __restrict__ cand_d) {
  __shared__ uint32_t hist[2048];
  __shared__ unsigned long long keys[kMaxC];
  __shared__ uint32_t ties[kTieCap];
  __shared__ uint32_t scratch[96];
  __shared__ uint32_t s_bin, s_below, s_nout, s_nties, s_total;
  const int q = blockIdx.x;
  const uint32_t kInfBits = 0x7F800000u;

  // ---- digit passes
  uint32_t prefix = 0;   // known high bits of the threshold
  int known = 0;         // number of known high bits
  uint32_t need = (uint32_t)C;
  uint32_t below_total = 0;
  const int shifts[3] = {21, 10, 0};
  const int widths[3] = {11, 11, 10};
  bool take_all = false;
  for (int pass = 0; pass < 3; ++pass) {
    const int nb = 1 << widths[pass];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int p = 0; p < nprobe; ++p) {
      SegIter it = seg_of(q, p, nprobe, probe, pair_of, pair_off, seg_base, blk_off, D);
      for (uint32_t i = threadIdx.x; i < it.len; i += blockDim.x) {
        uint32_t k = fkey(it.base[i]);
        if (k >= kInfBits) continue;
        if (known && (k >> (32 - known)) != prefix) continue;
        atomicAdd(&hist[(k >> shifts[pass]) & (nb - 1)], 1u);
      }
    }
    __syncthreads();
    if (pass == 0) {
      // total valid count
      uint32_t sum = 0;
      for (int i = threadIdx.x; i < nb; i += blockDim.x) sum += hist[i];
      uint32_t excl = block_exclusive_scan<uint32_t>(sum, &s_total, scratch);
      (void)excl;
      if (s_total <= need) {
        take_all = true;
        break;
      }
    }
    find_bin(hist, nb, need, &s_bin, &s_below, scratch);
    need -= s_below;
    below_total += s_below;
    prefix = (prefix << widths[pass]) | s_bin;
    known += widths[pass];
    __syncthreads();
  }
  const uint32_t T = take_all ? kInfBits : prefix;  // threshold key
  // ---- collect keys < T (all of them) and the ties == T
  if (threadIdx.x == 0) {
    s_nout = 0;
    s_nties = 0;
  }
  __syncthreads();
  for (int p = 0; p < nprobe; ++p) {
    SegIter it = seg_of(q, p, nprobe, probe, pair_of, pair_off, seg_base, blk_off, D);
    for (uint32_t i = threadIdx.x; i < it.len; i += blockDim.x) {
      uint32_t k = fkey(it.base[i]);
      if (k >= kInfBits) continue;
      uint32_t id = ids[it.row0 + i];
      if (k < T) {
        uint32_t pos = atomicAdd(&s_nout, 1u);
        if (pos < (uint32_t)kMaxC) keys[pos] = ((unsigned long long)k << 32) | id;
      } else if (k == T) {
        uint32_t pos = atomicAdd(&s_nties, 1u);
        if (pos < (uint32_t)kTieCap) ties[pos] = id;
      }
    }
  }
  __syncthreads();
  uint32_t nout = s_nout;
  if (!take_all) {
    const uint32_t need_eq = (uint32_t)C - nout;
    if (s_nties <= (uint32_t)kTieCap) {
      // smallest need_eq ids among the ties: bitonic on the tie ids
      const int nt = (int)s_nties;
      const int np2 = pow2_at_least(nt);
      __shared__ unsigned long long tk[kTieCap];
      for (int i = threadIdx.x; i < np2; i += blockDim.x) tk[i] = i < nt ? ties[i] : ~0ull;
      __syncthreads();
      bitonic_sort_u64(tk, np2);
      for (uint32_t i = threadIdx.x; i < need_eq; i += blockDim.x)
        keys[nout + i] = ((unsigned long long)T << 32) | (uint32_t)tk[i];
    } else {
      // degenerate: more ties than the buffer; take ids one at a time
      __shared__ uint32_t s_min;
      uint32_t last = 0;
      bool first = true;
      for (uint32_t e = 0; e < need_eq; ++e) {
        if (threadIdx.x == 0) s_min = 0xFFFFFFFFu;
        __syncthreads();
        uint32_t mine = 0xFFFFFFFFu;
        for (int p = 0; p < nprobe; ++p) {
          SegIter it = seg_of(q, p, nprobe, probe, pair_of, pair_off, seg_base, blk_off, D);
          for (uint32_t i = threadIdx.x; i < it.len; i += blockDim.x) {
            if (fkey(it.base[i]) != T) continue;
            uint32_t id = ids[it.row0 + i];
            if ((first || id > last) && id < mine) mine = id;
          }
        }
        atomicMin(&s_min, mine);
        __syncthreads();
        last = s_min;
        first = false;
        if (threadIdx.x == 0) keys[nout + e] = ((unsigned long long)T << 32) | last;
        __syncthreads();
      }
    }
    nout = (uint32_t)C;
  }
  __syncthreads();
  const int n2 = pow2_at_least(C);
  for (int i = threadIdx.x; i < n2; i += blockDim.x)
    if (i >= (int)nout) keys[i] = ~0ull;
  __syncthreads();
  bitonic_sort_u64(keys, n2);
  for (int i = threadIdx.x; i < C; i += blockDim.x) {
    unsigned long long kk = keys[i];
    bool ok = i < (int)nout;
    cand_id[(size_t)q * C + i] = ok ? (uint32_t)(kk & 0xFFFFFFFFu) : kInvalidId;
    cand_d[(size_t)q * C + i] = ok ? __uint_as_float((uint32_t)(kk >> 32)) : INFINITY;
  }
}

// ------------------------------------------------------------------ rerank

// One CTA per query: exact sum_t (q_t - x_t)^2 of every pool member (one warp
// per member, 16-byte loads of the raw row), then the k smallest (dist, id).
template <bool kBF16>
__global__ void __launch_bounds__(256) k_rerank(const float* __restrict__ Q, const void* __restrict__ Xv, int d,
                                                int C, int k, const uint32_t* __restrict__ cand_id,
                                                int64_t* __restrict__ out_ids, float* __restrict__ out_d) {
  extern __shared__ float sq[];  // [d]
  __shared__ unsigned long long keys[kMaxC];
  const int q = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = threadIdx.x; t < d; t += blockDim.x) sq[t] = Q[(size_t)q * d + t];
  __syncthreads();
  const int n2 = pow2_at_least(C);
  for (int c = warp; c < n2; c += 8) {
    unsigned long long key = ~0ull;
    uint32_t id = c < C ? cand_id[(size_t)q * C + c] : kInvalidId;
    if (id != kInvalidId) {
      float acc = 0.f;
      if (!kBF16) {
        const float* x = reinterpret_cast<const float*>(Xv) + (size_t)id * d;
        if ((d & 3) == 0) {
          for (int t = lane * 4; t < d; t += 128) {
            float4 v = __ldg(reinterpret_cast<const float4*>(x + t));
            float a0 = sq[t] - v.x, a1 = sq[t + 1] - v.y, a2 = sq[t + 2] - v.z, a3 = sq[t + 3] - v.w;
            acc = fmaf(a0, a0, acc);
            acc = fmaf(a1, a1, acc);
            acc = fmaf(a2, a2, acc);
            acc = fmaf(a3, a3, acc);
          }
        } else {
          for (int t = lane; t < d; t += 32) {
            float a0 = sq[t] - __ldg(x + t);
            acc = fmaf(a0, a0, acc);
          }
        }
      } else {
        const uint16_t* x = reinterpret_cast<const uint16_t*>(Xv) + (size_t)id * d;
        if ((d & 7) == 0) {
          for (int t = lane * 8; t < d; t += 256) {
            uint4 v = __ldg(reinterpret_cast<const uint4*>(x + t));
            uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              float lo = __uint_as_float(w[h] << 16), hi = __uint_as_float(w[h] & 0xFFFF0000u);
              float a0 = sq[t + 2 * h] - lo, a1 = sq[t + 2 * h + 1] - hi;
              acc = fmaf(a0, a0, acc);
              acc = fmaf(a1, a1, acc);
            }
          }
        } else {
          for (int t = lane; t < d; t += 32) {
            float a0 = sq[t] - __uint_as_float((uint32_t)__ldg(x + t) << 16);
            acc = fmaf(a0, a0, acc);
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      key = ((unsigned long long)__float_as_uint(acc) << 32) | id;
    }
    if (lane == 0) keys[c] = key;
  }
  __syncthreads();
  bitonic_sort_u64(keys, n2);
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    unsigned long long kk = i < n2 ? keys[i] : ~0ull;
    bool ok = kk != ~0ull;
    out_ids[(size_t)q * k + i] = ok ? (int64_t)(kk & 0xFFFFFFFFu) : -1;
    out_d[(size_t)q * k + i] = ok ? __uint_as_float((uint32_t)(kk >> 32)) : INFINITY;
  }
}

// ------------------------------------------------------------------ host side

// Makes the index's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

struct Ws {
  float* route_d;
  int32_t* probe;
  float* probe_d;
  uint32_t* gcnt;
  uint32_t* gcur;
  uint32_t* pair_off;
  uint64_t* seg_base;
  uint32_t* grp_off;
  uint32_t* pair_q;
  uint32_t* pair_of;
  float* zq;
  float* rhoq;
  float* D;
  uint32_t* cand_id;
  float* cand_d;
  size_t bytes;
};

Ws carve(const Index& I, uint32_t nq, uint32_t C, uint32_t nprobe, void* base) {
  Carver c(base);
  Ws w;
  const size_t P = (size_t)nq * nprobe;
  w.route_d = c.take<float>((size_t)nq * I.G);
  w.probe = c.take<int32_t>(P);
  w.probe_d = c.take<float>(P);
  w.gcnt = c.take<uint32_t>(I.G);
  w.gcur = c.take<uint32_t>(I.G);
  w.pair_off = c.take<uint32_t>(I.G + 1);
  w.seg_base = c.take<uint64_t>(I.G);
  w.grp_off = c.take<uint32_t>(I.G + 1);
  w.pair_q = c.take<uint32_t>(P);
  w.pair_of = c.take<uint32_t>(P);
  w.zq = c.take<float>(P * I.r);
  w.rhoq = c.take<float>(P);
  w.D = c.take<float>((size_t)nq * I.h_top_padded_prefix[nprobe]);
  w.cand_id = c.take<uint32_t>((size_t)nq * C);
  w.cand_d = c.take<float>((size_t)nq * C);
  w.bytes = align_up(c.off, 256);
  return w;
}

int check_params(const Index& I, uint32_t nq, uint32_t k, uint32_t& C, uint32_t nprobe) {
  if (k < 1) return fail(HNTL_EINVAL, "k must be >= 1");
  if (C < k) C = k;
  if (C > (uint32_t)kMaxC) return fail(HNTL_EINVAL, "C (after raising it to k) must be <= 1024");
  if (nprobe < 1 || nprobe > I.G) return fail(HNTL_EINVAL, "nprobe must be in [1, G]");
  if ((uint64_t)nq * nprobe >= (1ull << 31)) return fail(HNTL_EINVAL, "nq * nprobe too large");
  return HNTL_OK;
}

int launch_route(const Index& I, const float* Qd, uint32_t nq, uint32_t nprobe, const Ws& w, cudaStream_t st) {
  dim3 grid((I.G + kRT - 1) / kRT, (nq + kRT - 1) / kRT);
  k_route_dist<<<grid, 256, 0, st>>>(Qd, I.M, (int)nq, (int)I.G, (int)I.d, w.route_d);
  size_t smem = (size_t)kSelWarps * I.G * sizeof(float);
  static thread_local bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_route_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kSelWarps * kMaxG * (int)sizeof(float));
    attr_set = true;
  }
  k_route_select<<<(nq + kSelWarps - 1) / kSelWarps, kSelWarps * 32, smem, st>>>(w.route_d, (int)nq, (int)I.G,
                                                                                  (int)nprobe, w.probe, w.probe_d);
  HNTL_CUDA_TRY(cudaGetLastError());
  return HNTL_OK;
}

template <int RT>
void launch_scan(const Index& I, const Ws& w, const int64_t* filter, cudaStream_t st) {
  k_scan_fp32<RT><<<(unsigned)I.n_blocks, kBlockRows, 0, st>>>(
      I.blk_grain, I.blk_off, I.grain_rows, I.Zb, I.rho, I.attr_b, (int)I.r, w.gcnt, w.pair_off, w.seg_base,
      w.pair_q, w.zq, w.rhoq, filter, w.D);
}

// Stage timing: CUDA events recorded on the search's stream between stages.
using StageEvents = std::array<cudaEvent_t, HNTL_NSTAGES + 1>;
struct Profiler {
  std::mutex mu;
  bool on = false;
  std::vector<StageEvents> pending, pool;
};
Profiler& profiler() {
  static Profiler p;
  return p;
}
bool profile_begin(StageEvents& ev) {
  Profiler& P = profiler();
  std::lock_guard<std::mutex> lk(P.mu);
  if (!P.on) return false;
  if (!P.pool.empty()) {
    ev = P.pool.back();
    P.pool.pop_back();
    return true;
  }
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) return false;
  return true;
}
void profile_end(const StageEvents& ev) {
  Profiler& P = profiler();
  std::lock_guard<std::mutex> lk(P.mu);
  P.pending.push_back(ev);
}

}  // namespace

int search(const Index& I, const float* Qd, uint32_t nq, uint32_t k, uint32_t C, uint32_t nprobe,
           const int64_t* filter, void* ws, size_t ws_bytes, int64_t* out_ids, float* out_d, uint32_t* cand_ids,
           float* cand_d, int32_t* probe_out, cudaStream_t st) {
  int rc = check_params(I, nq, k, C, nprobe);
  if (rc) return rc;
  if (filter && !I.has_attr) return fail(HNTL_EINVAL, "filter given but the index has no attribute column");
  if (I.precision != HNTL_PREC_FP32) return fail(HNTL_EINVAL, "precision form search is not built yet");
  if (nq == 0) return HNTL_OK;
  if (!Qd || !ws || !out_ids || !out_d) return fail(HNTL_EINVAL, "null buffer");
  if ((cand_ids == nullptr) != (cand_d == nullptr)) return fail(HNTL_EINVAL, "pass both pool buffers or neither");
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(HNTL_EINVAL, "workspace must be 256-byte aligned");
  Ws w = carve(I, nq, C, nprobe, ws);
  if (ws_bytes < w.bytes) return fail(HNTL_EINVAL, "workspace too small");
  if (cand_ids) {
    w.cand_id = cand_ids;
    w.cand_d = cand_d;
  }
  DeviceGuard dg(I.device);
  if (!dg.ok) return fail(HNTL_ECUDA, "cannot make the index's device current");
  StageEvents ev;
  const bool prof = profile_begin(ev);
  auto mark = [&](int i) {
    if (prof) cudaEventRecord(ev[i], st);
  };
  mark(0);
  HNTL_CUDA_TRY(cudaMemsetAsync(w.gcnt, 0, sizeof(uint32_t) * I.G, st));
  HNTL_CUDA_TRY(cudaMemsetAsync(w.gcur, 0, sizeof(uint32_t) * I.G, st));
  if ((rc = launch_route(I, Qd, nq, nprobe, w, st))) return rc;
  mark(1);
  const int P = (int)(nq * nprobe);
  k_bucket_count<<<(P + 255) / 256, 256, 0, st>>>(w.probe, P, w.gcnt);
  k_bucket_scan<<<1, 1024, 0, st>>>(w.gcnt, I.blk_off, (int)I.G, w.pair_off, w.seg_base, w.grp_off);
  k_bucket_scatter<<<(P + 255) / 256, 256, 0, st>>>(w.probe, (int)nq, (int)nprobe, w.pair_off, w.gcur, w.pair_q,
                                                    w.pair_of);
  mark(2);
  {
    size_t smem = (size_t)kPairsPerGroup * I.d * sizeof(float);
    if (smem > 48 * 1024)
      HNTL_CUDA_TRY(cudaFuncSetAttribute(k_project, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    unsigned grid = (unsigned)std::min<size_t>((size_t)P / kPairsPerGroup + I.G, 148 * 16);
    k_project<<<grid, 256, smem, st>>>(Qd, I.M, I.U, (int)I.d, (int)I.r, (int)I.G, w.grp_off, w.pair_off, w.pair_q,
                                       w.zq, w.rhoq);
  }
  mark(3);
  if (I.r <= 8) launch_scan<8>(I, w, filter, st);
  else if (I.r <= 16) launch_scan<16>(I, w, filter, st);
  else if (I.r <= 32) launch_scan<32>(I, w, filter, st);
  else launch_scan<64>(I, w, filter, st);
  mark(4);
  k_select<<<nq, kSelThreads, 0, st>>>((int)nprobe, (int)C, w.probe, w.pair_of, w.pair_off, w.seg_base, I.blk_off,
                                       I.ids, w.D, w.cand_id, w.cand_d);
  mark(5);
  {
    size_t smem = (size_t)I.d * sizeof(float);
    if (smem > 40 * 1024) {
      HNTL_CUDA_TRY(cudaFuncSetAttribute(k_rerank<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    k_rerank<false><<<nq, 256, smem, st>>>(Qd, I.X, (int)I.d, (int)C, (int)k, w.cand_id, out_ids, out_d);
  }
  mark(6);
  if (prof) profile_end(ev);
  if (probe_out)
    HNTL_CUDA_TRY(cudaMemcpyAsync(probe_out, w.probe, sizeof(int32_t) * nq * nprobe, cudaMemcpyDeviceToDevice, st));
  HNTL_CUDA_TRY(cudaGetLastError());
  return HNTL_OK;
}

size_t workspace_bytes(const Index& I, uint32_t nq, uint32_t k, uint32_t C, uint32_t nprobe) {
  if (check_params(I, nq, k, C, nprobe)) return 0;
  return carve(I, nq, C, nprobe, nullptr).bytes;
}

int route_only(const Index& I, const float* Qd, uint32_t nq, uint32_t nprobe, void* ws, size_t ws_bytes,
               int32_t* probe, float* probe_d, cudaStream_t st) {
  uint32_t C = 1;
  int rc = check_params(I, nq, 1, C, nprobe);
  if (rc) return rc;
  if (nq == 0) return HNTL_OK;
  if (!Qd || !ws || !probe || !probe_d) return fail(HNTL_EINVAL, "null buffer");
  if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(HNTL_EINVAL, "workspace must be 256-byte aligned");
  Ws w = carve(I, nq, C, nprobe, ws);
  if (ws_bytes < w.bytes) return fail(HNTL_EINVAL, "workspace too small");
  w.probe = probe;
  w.probe_d = probe_d;
  DeviceGuard dg(I.device);
  if (!dg.ok) return fail(HNTL_ECUDA, "cannot make the index's device current");
  return launch_route(I, Qd, nq, nprobe, w, st);
}

}  // namespace hntl

extern "C" {

int hntl_profile_enable(int on) {
  hntl::clear_error();
  hntl::Profiler& P = hntl::profiler();
  std::lock_guard<std::mutex> lk(P.mu);
  P.on = on != 0;
  return HNTL_OK;
}

int hntl_profile_read(double* ms, uint64_t* calls) {
  hntl::clear_error();
  if (!ms || !calls) return hntl::fail(HNTL_EINVAL, "null argument");
  hntl::Profiler& P = hntl::profiler();
  std::lock_guard<std::mutex> lk(P.mu);
  for (int s = 0; s < HNTL_NSTAGES; ++s) ms[s] = 0.0;
  *calls = 0;
  for (auto& ev : P.pending) {
    HNTL_CUDA_TRY(cudaEventSynchronize(ev[HNTL_NSTAGES]));
    for (int s = 0; s < HNTL_NSTAGES; ++s) {
      float t = 0.f;
      HNTL_CUDA_TRY(cudaEventElapsedTime(&t, ev[s], ev[s + 1]));
      ms[s] += t;
    }
    ++*calls;
    P.pool.push_back(ev);
  }
  P.pending.clear();
  return HNTL_OK;
}

size_t hntl_search_workspace_bytes(const hntl_index* idx, uint32_t nq, uint32_t k, uint32_t C, uint32_t nprobe) {
  hntl::clear_error();
  if (!idx) {
    hntl::fail(HNTL_EINVAL, "null index");
    return 0;
  }
  return hntl::workspace_bytes(idx->I, nq, k, C, nprobe);
}

int hntl_search(const hntl_index* idx, const float* d_queries, uint32_t nq, uint32_t k, uint32_t C, uint32_t nprobe,
                const int64_t* d_filter, void* d_ws, size_t ws_bytes, int64_t* d_out_ids, float* d_out_dist,
                uint32_t* d_cand_ids, float* d_cand_dist, int32_t* d_probe, void* stream) {
  hntl::clear_error();
  if (!idx) return hntl::fail(HNTL_EINVAL, "null index");
  return hntl::search(idx->I, d_queries, nq, k, C, nprobe, d_filter, d_ws, ws_bytes, d_out_ids, d_out_dist,
                      d_cand_ids, d_cand_dist, d_probe, static_cast<cudaStream_t>(stream));
}

int hntl_route(const hntl_index* idx, const float* d_queries, uint32_t nq, uint32_t nprobe, void* d_ws,
               size_t ws_bytes, int32_t* d_probe, float* d_probe_dist, void* stream) {
  hntl::clear_error();
  if (!idx) return hntl::fail(HNTL_EINVAL, "null index");
  return hntl::route_only(idx->I, d_queries, nq, nprobe, d_ws, ws_bytes, d_probe, d_probe_dist,
                          static_cast<cudaStream_t>(stream));
}

size_t hntl_search_host_workspace_bytes(const hntl_index* idx, uint32_t nq, uint32_t k, uint32_t C, uint32_t nprobe,
                                        int with_filter) {
  hntl::clear_error();
  if (!idx) {
    hntl::fail(HNTL_EINVAL, "null index");
    return 0;
  }
  size_t need = hntl::workspace_bytes(idx->I, nq, k, C, nprobe);
  if (need == 0) return 0;
  hntl::Carver c(nullptr);
  c.take<float>((size_t)nq * idx->I.d);
  if (with_filter) c.take<int64_t>((size_t)nq * 2);
  c.take<int64_t>((size_t)nq * k);
  c.take<float>((size_t)nq * k);
  return need + hntl::align_up(c.off, 256);
}

int hntl_search_host(const hntl_index* idx, const float* h_queries, uint32_t nq, uint32_t k, uint32_t C,
                     uint32_t nprobe, const int64_t* h_filter, void* d_ws, size_t ws_bytes, int64_t* h_out_ids,
                     float* h_out_dist, void* stream) {
  hntl::clear_error();
  if (!idx) return hntl::fail(HNTL_EINVAL, "null index");
  const hntl::Index& I = idx->I;
  if (nq == 0) return HNTL_OK;
  if (!h_queries || !h_out_ids || !h_out_dist || !d_ws) return hntl::fail(HNTL_EINVAL, "null buffer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // device staging for queries, filters and results follows the search workspace
  size_t need = hntl::workspace_bytes(I, nq, k, C, nprobe);
  if (need == 0) return HNTL_EINVAL;
  hntl::Carver c(static_cast<char*>(d_ws) + need);
  float* dQ = c.take<float>((size_t)nq * I.d);
  int64_t* dF = h_filter ? c.take<int64_t>((size_t)nq * 2) : nullptr;
  int64_t* dI = c.take<int64_t>((size_t)nq * k);
  float* dD = c.take<float>((size_t)nq * k);
  size_t total = need + hntl::align_up(c.off, 256);
  if (ws_bytes < total) return hntl::fail(HNTL_EINVAL, "workspace too small for the host form");
  HNTL_CUDA_TRY(cudaMemcpyAsync(dQ, h_queries, sizeof(float) * nq * I.d, cudaMemcpyHostToDevice, st));
  if (dF) HNTL_CUDA_TRY(cudaMemcpyAsync(dF, h_filter, sizeof(int64_t) * nq * 2, cudaMemcpyHostToDevice, st));
  int rc = hntl::search(I, dQ, nq, k, C, nprobe, dF, d_ws, need, dI, dD, nullptr, nullptr, nullptr, st);
  if (rc) return rc;
  HNTL_CUDA_TRY(cudaMemcpyAsync(h_out_ids, dI, sizeof(int64_t) * nq * k, cudaMemcpyDeviceToHost, st));
  HNTL_CUDA_TRY(cudaMemcpyAsync(h_out_dist, dD, sizeof(float) * nq * k, cudaMemcpyDeviceToHost, st));
  HNTL_CUDA_TRY(cudaStreamSynchronize(st));
  return HNTL_OK;
}

}  // extern "C"
