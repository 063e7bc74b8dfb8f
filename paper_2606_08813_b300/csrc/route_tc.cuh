// Centroid routing on the tensor cores (sec. 2.1 step 1, sec. 2.3 item 1).
//
// k_route_tc: S = Q M^T on tcgen05 (TF32 for FP32 indices, BF16 for the
// precision form; FP32 accumulation in TMEM), persistent and
// warp-specialised: operands streamed by TMA through a 4-stage shared-memory
// ring, two TMEM accumulators so that the epilogue of one 128-query x
// 256-centre tile (the approximate squared distance ||q||^2 + ||mu||^2 -
// 2 q.mu) overlaps the MMAs of the next.
//
// k_route_refine: the approximate distance is within
//   m(q, g) = eps_dot ||q|| ||mu_g|| + eps_norm (||q||^2 + ||mu_g||^2)
// of the exact one (route_margin() sets both, with a factor 2 of safety):
//   eps_dot, the dot product: TF32 operands are each rounded by at most
//     2^-10 relative, so a product by 2^-9 of |q_t mu_t|, summed at most
//     2^-9 ||q|| ||mu|| (Cauchy-Schwarz), doubled in the distance; BF16
//     operands multiply exactly, so only the FP32 accumulation remains: at
//     most K/16 + 16 roundings of 2^-23 (groups of 16 products added to the
//     accumulator, and within a group), of sum |q_t mu_t| <= ||q|| ||mu||;
//   eps_norm, the squared norms (one warp each: d/32 sequential additions per
//     lane, five butterfly levels) and the final sum (||q||^2 + ||mu||^2 - 2S).
// With U the nprobe-th smallest approx + margin, any centre whose approx -
// margin exceeds U cannot be among the nprobe nearest, so only the others
// (typically nprobe plus a few) get their exact direct-form distance sum
// (q_t - mu_t)^2, and the nprobe smallest (distance, grain) are kept: the same
// selection as the direct-form routing, at a fraction of its arithmetic.
#pragma once

#include <cuda_bf16.h>

#include "hntl_internal.cuh"
#include "kernels_common.cuh"
#include "tc_common.cuh"

namespace hntl {
namespace {

constexpr int kRTM = 128, kRTN = 256, kRStages = 4;
constexpr int kRThreads = 192;  // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr int kRouteTcSmem = kRStages * (kRTM + kRTN) * 128 + 1024;

// Persistent, warp-specialised: CTA b takes the 128-query x 256-centre tiles
// b, b + grid, ... (centre blocks vary fastest, so CTAs working at the same
// time share their query tile in L2).
//   warp 0     one thread streams each tile's K blocks (query and centre
//              rows, 128 bytes of K each) by TMA through the stage ring.
//   warp 1     one thread issues the MMAs of a tile into one of two TMEM
//              accumulators (256 columns each) and hands it on through `accf`.
//   warps 2-5  epilogue, warp w for TMEM lane quarter w % 4: reads its 32
//              rows of the finished accumulator, frees it through `acce`, and
//              writes ||q||^2 + ||mu||^2 - 2 q.mu while the next tile's MMAs run.
template <bool kBF16>
__global__ void __launch_bounds__(kRThreads, 1) k_route_tc(const __grid_constant__ CUtensorMap mapQ,
                                                        const __grid_constant__ CUtensorMap mapM, int nq, int G,
                                                        int d, const float* __restrict__ qn,
                                                        const float* __restrict__ mn, float* __restrict__ Dt,
                                                        int* __restrict__ err) {
  constexpr int S = kRStages;
  constexpr int kElem = kBF16 ? 2 : 4;
  constexpr int kKB = 128 / kElem;       // K elements per stage (one 128-byte row)
  constexpr int kStep = kBF16 ? 16 : 8;  // K per MMA
  constexpr uint32_t kBytesA = kRTM * 128, kBytesB = kRTN * 128;
  constexpr uint32_t kIdesc = tc::idesc_f32acc(kBF16 ? 1u : 2u, kRTM, kRTN);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[S], empty[S], accf[2], acce[2], fin;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  __shared__ uint32_t s_it_prod, s_it_mma;  // K blocks loaded by the producer / consumed by the MMA thread
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::tmem_alloc(&tmem_base, 2 * kRTN);
  if (tid == 32) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(&accf[a], 1);
      tc::mbar_init(&acce[a], 4);
    }
    tc::mbar_init(&fin, 1);
    tc::mbar_fence_init();
    s_fail = 0;
    s_it_prod = s_it_mma = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const int n_gb = (G + kRTN - 1) / kRTN;
  const int total = n_gb * ((nq + kRTM - 1) / kRTM);
  const int nkb = (d + kKB - 1) / kKB;
  if (warp == 0) {
    if (lane == 0) {  // producer
      uint32_t it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
        const int q0 = (t / n_gb) * kRTM, g0 = (t % n_gb) * kRTN;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % S);
          if (it >= (uint32_t)S && !tc::mbar_wait(&empty[s], ((it / S) - 1) & 1)) {
            ok = false;
            break;
          }
          uint8_t* sa = smem + s * (kBytesA + kBytesB);
          tc::mbar_expect_tx(&full[s], kBytesA + kBytesB);
          tc::tma_load_2d(&mapQ, &full[s], sa, kb * kKB, q0);
          tc::tma_load_2d(&mapM, &full[s], sa + kBytesA, kb * kKB, g0);
        }
      }
      s_it_prod = it;
      if (!ok) atomicExch(&s_fail, 1);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issue
      uint32_t it = 0, li = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++li) {
        const int a = (int)(li & 1);
        if (li >= 2 && !tc::mbar_wait(&acce[a], ((li >> 1) - 1) & 1)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t acc = tmem + (uint32_t)(a * kRTN);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = (int)(it % S);
          if (!tc::mbar_wait(&full[s], (it / S) & 1)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_u32(smem + s * (kBytesA + kBytesB));
#pragma unroll
          for (int ks = 0; ks < kKB / kStep; ++ks)
            tc::mma<kBF16>(acc, tc::desc_sw128(sa + ks * 32), tc::desc_sw128(sa + kBytesA + ks * 32), kIdesc,
                           (kb | ks) != 0);
          tc::mma_commit(&empty[s]);
        }
        if (ok) tc::mma_commit(&accf[a]);
      }
      s_it_mma = it;
      if (!ok) atomicExch(&s_fail, 1);
      if (it > 0) {
        tc::mma_commit(&fin);  // arrives once every MMA issued above has completed
        if (!tc::mbar_wait(&fin, 0)) atomicExch(&s_fail, 1);
      }
    }
    __syncwarp();
  } else {
    // epilogue: TMEM lane quarter j = rows 32 j .. 32 j + 31 of each tile
    const int j = warp & 3;
    const bool vec = (G & 3) == 0;  // rows of Dt start on 16-byte boundaries
    bool failed = false;
    uint32_t li = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x, ++li) {
      const int a = (int)(li & 1);
      const int q0 = (t / n_gb) * kRTM, g0 = (t % n_gb) * kRTN;
      const int q = q0 + j * 32 + lane;
      const float qv = q < nq ? qn[q] : 0.f;
      if (__any_sync(0xffffffffu, !tc::mbar_wait(&accf[a], (li >> 1) & 1))) {  // warp-uniform
        failed = true;
        break;
      }
      tc::fence_after_sync();
#pragma unroll 1
      for (int c0 = 0; c0 < kRTN; c0 += 32) {
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(j * 32) << 16) + (uint32_t)(a * kRTN + c0), v);
        if (c0 + 32 == kRTN) {  // every column of this accumulator is in registers: free it
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&acce[a]);
        }
        const float mv = g0 + c0 + lane < G ? mn[g0 + c0 + lane] : 0.f;  // ||mu||^2 of column c0 + lane
        float* out = Dt + (size_t)q * G + g0 + c0;
        const int lim = G - (g0 + c0);  // columns of this chunk inside the matrix
#pragma unroll
        for (int c = 0; c < 32; c += 4) {
          const float m0 = __shfl_sync(0xffffffffu, mv, c), m1 = __shfl_sync(0xffffffffu, mv, c + 1);
          const float m2 = __shfl_sync(0xffffffffu, mv, c + 2), m3 = __shfl_sync(0xffffffffu, mv, c + 3);
          if (q < nq) {
            float4 o;
            o.x = (qv + m0) - 2.f * v[c];
            o.y = (qv + m1) - 2.f * v[c + 1];
            o.z = (qv + m2) - 2.f * v[c + 2];
            o.w = (qv + m3) - 2.f * v[c + 3];
            if (vec && c + 4 <= lim) {
              *reinterpret_cast<float4*>(out + c) = o;
            } else {
              if (c < lim) out[c] = o.x;
              if (c + 1 < lim) out[c + 1] = o.y;
              if (c + 2 < lim) out[c + 2] = o.z;
              if (c + 3 < lim) out[c + 3] = o.w;
            }
          }
        }
      }
    }
    if (failed) atomicExch(&s_fail, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid == 0 && s_fail) {
    // loads issued but never waited for (a wait gave up): let them land before the CTA exits
    for (uint32_t i = s_it_mma; i < s_it_prod; ++i) tc::mbar_wait(&full[i % S], (i / S) & 1, 1u << 16);
    atomicOr(err, tc::kErrTimeout);
  }
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 2 * kRTN);
  }
}

__device__ __forceinline__ uint32_t ordered_key(float x) {  // monotone map of any float (NaN -> top) to uint32
  if (!(x == x)) return 0xFFFFFFFFu;
  const uint32_t b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

constexpr int kRefineThreads = 256;
constexpr int kRefineCap = 1024;

constexpr int kRefineSmemMax = (8192 + 2 * kMaxG) * 4;  // d <= 8192 on this path

// Dynamic shared memory of k_route_refine: the query row and one or two key arrays.
inline size_t refine_smem_bytes(int d, int G, int nprobe) {
  return ((size_t)d + (nprobe > kRefineThreads ? 2 : 1) * (size_t)G) * sizeof(float);
}

// Margin coefficients of the refine shortlist (see the file header), with a
// factor 2 of safety: {eps_dot, eps_norm}.
inline void route_margin(bool bf16, int d, float* eps_dot, float* eps_norm) {
  const double u23 = 1.0 / 8388608.0;  // 2^-23
  const double dot = bf16 ? 2.0 * ((d + 15) / 16 + 16) * u23 : 2.0 * (2.0 / 512.0 + ((d + 15) / 16 + 16) * u23);
  const double norm = 2.0 * (((d + 31) / 32 + 6) * 0.5 * u23 + u23);
  *eps_dot = (float)dot;
  *eps_norm = (float)norm;
}

// ||q - mu_g||^2 in the direct form, one warp (the result in every lane). Each
// lane sums its elements in a fixed order (with rows of at most 1024 values
// and 16-byte strides: chunks of 8 (BF16) or 4 (FP32) consecutive values, all
// loads issued before use; else lane-strided), then a butterfly adds the
// lanes. Every kernel that forms a routing distance calls this, so a distance
// is bitwise the same whoever computed it. qv(t) is the query value (already
// BF16-rounded in the precision form).
template <bool kBF16, class QV>
__device__ __forceinline__ float warp_center_dist2(QV qv, const float* __restrict__ M,
                                                   const uint16_t* __restrict__ Mh, int g, int d, int lane) {
  float acc = 0.f;
  if (kBF16 && (d & 7) == 0 && d <= 1024) {
    const uint16_t* row = Mh + (size_t)g * d;
    uint4 v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int t = lane * 8 + 256 * i;
      v[i] = t < d ? __ldg(reinterpret_cast<const uint4*>(row + t)) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int t = lane * 8 + 256 * i;
      if (t < d) {
        const uint32_t w[4] = {v[i].x, v[i].y, v[i].z, v[i].w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const float a0 = qv(t + 2 * h) - __uint_as_float(w[h] << 16);
          const float a1 = qv(t + 2 * h + 1) - __uint_as_float(w[h] & 0xFFFF0000u);
          acc = fmaf(a0, a0, acc);
          acc = fmaf(a1, a1, acc);
        }
      }
    }
  } else if (!kBF16 && (d & 3) == 0 && d <= 1024) {
    const float* row = M + (size_t)g * d;
    float4 v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int t = lane * 4 + 128 * i;
      v[i] = t < d ? __ldg(reinterpret_cast<const float4*>(row + t)) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int t = lane * 4 + 128 * i;
      if (t < d) {
        const float a0 = qv(t) - v[i].x, a1 = qv(t + 1) - v[i].y, a2 = qv(t + 2) - v[i].z, a3 = qv(t + 3) - v[i].w;
        acc = fmaf(a0, a0, acc);
        acc = fmaf(a1, a1, acc);
        acc = fmaf(a2, a2, acc);
        acc = fmaf(a3, a3, acc);
      }
    }
  } else {
    for (int t = lane; t < d; t += 32) {
      const float m = kBF16 ? __uint_as_float((uint32_t)Mh[(size_t)g * d + t] << 16) : M[(size_t)g * d + t];
      const float df = qv(t) - m;
      acc = fmaf(df, df, acc);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

// Ascending bitonic sort of 64 keys held by one warp, key i in lane i % 32
// (a for i < 32, b above); stage j = 32 compares a lane's own two keys.
__device__ __forceinline__ void warp_sort64(unsigned long long& a, unsigned long long& b, int lane) {
#pragma unroll
  for (int k = 2; k <= 64; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j == 32) {
        const unsigned long long lo = a < b ? a : b, hi = a < b ? b : a;
        a = lo;
        b = hi;
      } else {
        const unsigned long long oa = __shfl_xor_sync(0xffffffffu, a, j), ob = __shfl_xor_sync(0xffffffffu, b, j);
        const bool lower = (lane & j) == 0;
        const bool up_a = (lane & k) == 0, up_b = ((lane + 32) & k) == 0;
        a = (lower == up_a) ? (oa < a ? oa : a) : (oa > a ? oa : a);
        b = (lower == up_b) ? (ob < b ? ob : b) : (ob > b ? ob : b);
      }
    }
  }
}

// One CTA per query: margin shortlist over the approximate distances, exact
// direct-form distances of the shortlist, the nprobe smallest (distance, g);
// with gcnt, each probe also counts one pair of its grain (the bucket
// stage's count, taken here while the kernel waits on memory anyway).
// In the precision form q and the centres are BF16 values (Mh).
template <bool kBF16>
__global__ void __launch_bounds__(kRefineThreads) k_route_refine(const float* __restrict__ Q, const float* __restrict__ M,
                                                                 const uint16_t* __restrict__ Mh,
                                                                 const float* __restrict__ qn,
                                                                 const float* __restrict__ mn,
                                                                 const float* __restrict__ Dt, int G, int d,
                                                                 int nprobe, float eps_dot, float eps_norm,
                                                                 int32_t* __restrict__ probe,
                                                                 float* __restrict__ probe_d,
                                                                 uint32_t* __restrict__ gcnt) {
  // dynamic: [d] query (BF16-rounded in the precision form), then the ordered
  // keys of approx + margin and approx - margin of every centre ([G] each), so
  // the row of approximate distances is read from memory once
  extern __shared__ float sq[];
  __shared__ uint32_t hist[256];
  __shared__ unsigned long long keys[kRefineCap];
  __shared__ uint32_t scratch[96];
  __shared__ uint32_t s_bin, s_below, s_cnt;
  const int q = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int t = threadIdx.x; t < d; t += blockDim.x) {
    float v = Q[(size_t)q * d + t];
    if (kBF16) v = __bfloat162float(__float2bfloat16_rn(v));
    sq[t] = v;
  }
  const float qv = qn[q];
  const float* Dq = Dt + (size_t)q * G;
  // khi is only kept for the radix path (nprobe > blockDim.x); the host sizes
  // the dynamic memory to match (refine_smem_bytes)
  const bool keep_hi = nprobe > (int)blockDim.x;
  uint32_t* khi = reinterpret_cast<uint32_t*>(sq + d);
  uint32_t* klo = keep_hi ? khi + G : khi;
  uint32_t my_min = 0xFFFFFFFFu;  // this thread's smallest approx + margin
  constexpr int kChunk = 8;        // loads of a thread issued together
  for (int g0 = threadIdx.x; g0 < G; g0 += kChunk * blockDim.x) {
    float Dv[kChunk], mv[kChunk];
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      const int g = g0 + u * blockDim.x;
      Dv[u] = g < G ? Dq[g] : 0.f;
      mv[u] = g < G ? mn[g] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      const int g = g0 + u * blockDim.x;
      if (g < G) {
        const float m = eps_dot * sqrtf(qv * mv[u]) + eps_norm * (qv + mv[u]);
        const uint32_t hi = ordered_key(Dv[u] + m);
        if (keep_hi) khi[g] = hi;
        klo[g] = ordered_key(Dv[u] - m);
        my_min = min(my_min, hi);
      }
    }
  }
  // U: any upper bound on the nprobe-th smallest approx + margin keeps the shortlist
  // exact. The nprobe-th smallest of the threads' minima is one (a subset's order
  // statistic is at least the full set's) and is rarely above the true one. Each
  // warp sorts its lanes' minima; the nprobe-th value of the union is found by
  // ranking every value against the other warps' sorted runs.
  uint32_t prefix = 0;
  bool have_u = false;
  if (nprobe <= (int)blockDim.x) {
    uint32_t v = my_min;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
        const uint32_t o = __shfl_xor_sync(0xffffffffu, v, j);
        const bool up = (lane & k) == 0, lower = (lane & j) == 0;
        v = (lower == up) ? min(v, o) : max(v, o);
      }
    }
    uint32_t* lists = reinterpret_cast<uint32_t*>(keys);  // nw sorted runs of 32
    lists[warp * 32 + lane] = v;
    __syncthreads();
    {  // U = the value of rank nprobe - 1 in the union of the runs, ties ordered by run
      // then position; each thread ranks its own value by a binary search of
      // every other run, and the one thread of that rank publishes it
      uint32_t rank = (uint32_t)lane;  // its own run: the lanes before it
      for (int w2 = 0; w2 < nw; ++w2) {
        if (w2 == warp) continue;
        const uint32_t* run = lists + w2 * 32;
        const bool before = w2 < warp;  // equal values of earlier runs rank lower
        int pos = 0;  // how many of run[] rank below v (a prefix of the sorted run)
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const uint32_t e = run[pos + step - 1];
          if (before ? e <= v : e < v) pos += step;
        }
        if (pos < 32 && (before ? run[pos] <= v : run[pos] < v)) ++pos;
        rank += (uint32_t)pos;
      }
      if (rank == (uint32_t)(nprobe - 1)) s_bin = v;
    }
    __syncthreads();
    prefix = s_bin;
    have_u = true;
    __syncthreads();  // the key runs are reused below
  } else {
    __syncthreads();
  }
  // else: U = nprobe-th smallest of approx + margin exactly (four 8-bit radix digits on ordered keys)
  uint32_t need = (uint32_t)nprobe;
  int known = 0;
  for (int pass = 0; pass < 4 && !have_u; ++pass) {
    const int sh = 24 - 8 * pass;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
      const uint32_t k = khi[g];
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
  const uint32_t Ukey = prefix;
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  for (int g = threadIdx.x; g < G; g += blockDim.x) {
    if (klo[g] <= Ukey) {
      const uint32_t pos = atomicAdd(&s_cnt, 1u);
      if (pos < (uint32_t)kRefineCap) keys[pos] = (unsigned long long)g;
    }
  }
  __syncthreads();
  const uint32_t cnt = s_cnt;
  const bool all = cnt > (uint32_t)kRefineCap;  // shortlist too long: fall back to every centre
  const int n = all ? G : (int)cnt;
  // exact distances, one warp per candidate; results are kept in the key list
  // (all == true: the first kRefineCap slots hold the running best, merged below)
  auto exact = [&](int g) {
    float acc = warp_center_dist2<kBF16>([&](int t) { return sq[t]; }, M, Mh, g, d, lane);
    if (!(acc == acc)) acc = INFINITY;
    return ((unsigned long long)__float_as_uint(acc) << 32) | (uint32_t)g;
  };
  if (!all) {
    for (int i = warp; i < n; i += nw) {
      const unsigned long long k = exact((int)(keys[i] & 0xFFFFFFFFu));
      if (lane == 0) keys[i] = k;
    }
    __syncthreads();
    if (n <= 64) {  // the usual case: one warp sorts, no block barriers
      if (warp == 0) {
        unsigned long long a = lane < n ? keys[lane] : ~0ull, b = lane + 32 < n ? keys[lane + 32] : ~0ull;
        warp_sort64(a, b, lane);
        keys[lane] = a;
        keys[lane + 32] = b;
      }
      __syncthreads();
    } else {
      const int n2 = pow2_at_least(n);
      for (int i = threadIdx.x; i < n2; i += blockDim.x)
        if (i >= n) keys[i] = ~0ull;
      __syncthreads();
      bitonic_sort_u64(keys, n2);
    }
  } else {
    // rare: exact distances of all G centres, nprobe rounds of a block-wide minimum above the last pick
    __shared__ unsigned long long s_best;
    unsigned long long last = 0;
    for (int p = 0; p < nprobe; ++p) {
      if (threadIdx.x == 0) s_best = ~0ull;
      __syncthreads();
      unsigned long long mine = ~0ull;
      for (int g = warp; g < G; g += nw) {
        const unsigned long long k = exact(g);
        if ((p == 0 || k > last) && k < mine) mine = k;
      }
      if (lane == 0) atomicMin(&s_best, mine);
      __syncthreads();
      last = s_best;
      if (threadIdx.x == 0) keys[p] = last;
      __syncthreads();
    }
  }
  for (int p = threadIdx.x; p < nprobe; p += blockDim.x) {
    const unsigned long long k = keys[p];
    probe[(size_t)q * nprobe + p] = (int32_t)(k & 0xFFFFFFFFu);
    probe_d[(size_t)q * nprobe + p] = __uint_as_float((uint32_t)(k >> 32));
    if (gcnt) atomicAdd(&gcnt[k & 0xFFFFFFFFu], 1u);  // the bucket stage's per-grain pair count
  }
}

// ||row||^2 of each row (FP32), one warp per row; BF16-rounded values when kBF16.
template <bool kBF16>
__global__ void k_row_norms(const float* __restrict__ X, int n, int d, float* __restrict__ out) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= n) return;
  float acc = 0.f;
  for (int t = lane; t < d; t += 32) {
    float v = X[(size_t)w * d + t];
    if (kBF16) v = __bfloat162float(__float2bfloat16_rn(v));
    acc = fmaf(v, v, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[w] = acc;
}

// The precision form's query preparation in one pass, one warp per row
// (d % 8 == 0): the BF16 copy of the row (round to nearest even) and the
// squared norm of the rounded values. Lane l takes the 8 values at
// 8 l + 256 j, j = 0, 1, ..., and adds their squares in that order: d / 32
// sequential additions per lane, then five butterfly levels, the rounding the
// routing margin allows for (as k_row_norms, in another order of the values).
__global__ void k_query_bf16(const float* __restrict__ X, int n, int d, uint16_t* __restrict__ out,
                             float* __restrict__ nrm) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= n) return;
  const float* x = X + (size_t)w * d;
  uint16_t* o = out + (size_t)w * d;
  float acc = 0.f;
#pragma unroll 4
  for (int t = lane * 8; t < d; t += 256) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(x + t));
    const float4 b = __ldg(reinterpret_cast<const float4*>(x + t + 4));
    const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint32_t pk[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const __nv_bfloat162 p2 = __floats2bfloat162_rn(v[2 * h], v[2 * h + 1]);  // .x low half, .y high half
      pk[h] = *reinterpret_cast<const uint32_t*>(&p2);
      const float lo = __uint_as_float(pk[h] << 16), hi = __uint_as_float(pk[h] & 0xFFFF0000u);
      acc = fmaf(lo, lo, acc);
      acc = fmaf(hi, hi, acc);
    }
    *reinterpret_cast<uint4*>(o + t) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  }
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o2);
  if (lane == 0) nrm[w] = acc;
}

// BF16 copy of FP32 rows (round to nearest even).
__global__ void k_to_bf16_rows(const float* __restrict__ X, size_t n, uint16_t* __restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __bfloat16_as_ushort(__float2bfloat16_rn(X[i]));
}

// -bf16(x): the sign bit of the rounded value flipped (exact)
__global__ void k_to_bf16_rows_neg(const float* __restrict__ X, size_t n, uint16_t* __restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (uint16_t)(__bfloat16_as_ushort(__float2bfloat16_rn(X[i])) ^ 0x8000u);
}

}  // namespace
}  // namespace hntl
