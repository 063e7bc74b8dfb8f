// Exact rerank of the pool (sec. 2.1 step 4, Mode B): sum_t (q_t - x_t)^2
// of every pool member against the FP32 query, the k smallest (dist, id).
#pragma once

#include "hntl_internal.cuh"
#include "kernels_common.cuh"

namespace hntl {
namespace {

// One CTA per query: exact sum_t (q_t - x_t)^2 of every pool member (one warp
// per member, 16-byte loads of the raw row), then the k smallest (dist, id).
// kRefine (BF16 rows with their second parts Xl = bf16(x - bf16(x))): the
// min(C, 2k) smallest of that ranking are scored again against
// bf16(x) + xl (exact in FP32: 16 significant bits) and the k smallest of
// those are returned.
template <bool kBF16, bool kRefine = false>
__global__ void __launch_bounds__(256) k_rerank(const float* __restrict__ Q, const void* __restrict__ Xv, int d,
                                                int C, int k, const uint32_t* __restrict__ cand_id,
                                                int64_t* __restrict__ out_ids, float* __restrict__ out_d,
                                                const uint32_t* __restrict__ qk, const uint32_t* __restrict__ qC,
                                                const uint16_t* __restrict__ Xl = nullptr) {
  extern __shared__ float sq[];  // [d]
  __shared__ unsigned long long keys[kMaxC];
  const int q = blockIdx.x;
  const uint32_t* cid = cand_id + (size_t)q * C;  // rows C (the batch's largest pool) apart
  int64_t* oid = out_ids + (size_t)q * k;         // rows k (the batch's largest k) apart
  float* od = out_d + (size_t)q * k;
  if (qC) {  // mixed batch: this query's own pool size and result count
    const int kq = (int)qk[q];
    for (int i = kq + threadIdx.x; i < k; i += blockDim.x) {
      oid[i] = -1;
      od[i] = INFINITY;
    }
    C = (int)qC[q];
    k = kq;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = threadIdx.x; t < d; t += blockDim.x) sq[t] = Q[(size_t)q * d + t];
  __syncthreads();
  const int n2 = pow2_at_least(C);
  // BF16 rows of up to 1024 values: two candidates a warp at a time, the two
  // rows' 16-byte loads issued interleaved before the sums (six loads of 512
  // bytes per warp in flight at d = 768, as many as one FP32 row gives; three
  // or four rows a warp, the two rows' loads one row after the other, and
  // this loop in the refined rerank's first stage measured slower)
  if (kBF16 && !kRefine && (d & 7) == 0 && d <= 1024) {
    for (int c = warp; c < n2; c += 16) {
      const int c2 = c + 8;
      const uint32_t ida = c < C ? cid[c] : kInvalidId, idb = c2 < C && c2 < n2 ? cid[c2] : kInvalidId;
      const uint16_t* xa = reinterpret_cast<const uint16_t*>(Xv) + (size_t)(ida != kInvalidId ? ida : 0) * d;
      const uint16_t* xb = reinterpret_cast<const uint16_t*>(Xv) + (size_t)(idb != kInvalidId ? idb : 0) * d;
      uint4 va[4], vb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int t = lane * 8 + 256 * i;
        va[i] = (ida != kInvalidId && t < d) ? __ldg(reinterpret_cast<const uint4*>(xa + t)) : make_uint4(0, 0, 0, 0);
        vb[i] = (idb != kInvalidId && t < d) ? __ldg(reinterpret_cast<const uint4*>(xb + t)) : make_uint4(0, 0, 0, 0);
      }
      float acca = 0.f, accb = 0.f;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int t = lane * 8 + 256 * i;
        if (t < d) {
          const uint32_t wa[4] = {va[i].x, va[i].y, va[i].z, va[i].w}, wb[4] = {vb[i].x, vb[i].y, vb[i].z, vb[i].w};
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const float q0 = sq[t + 2 * h], q1 = sq[t + 2 * h + 1];
            const float a0 = q0 - __uint_as_float(wa[h] << 16), a1 = q1 - __uint_as_float(wa[h] & 0xFFFF0000u);
            const float b0 = q0 - __uint_as_float(wb[h] << 16), b1 = q1 - __uint_as_float(wb[h] & 0xFFFF0000u);
            acca = fmaf(a0, a0, acca);
            acca = fmaf(a1, a1, acca);
            accb = fmaf(b0, b0, accb);
            accb = fmaf(b1, b1, accb);
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        acca += __shfl_xor_sync(0xffffffffu, acca, o);
        accb += __shfl_xor_sync(0xffffffffu, accb, o);
      }
      if (lane == 0) {
        keys[c] = ida != kInvalidId ? ((unsigned long long)__float_as_uint(acca) << 32) | ida : ~0ull;
        if (c2 < n2) keys[c2] = idb != kInvalidId ? ((unsigned long long)__float_as_uint(accb) << 32) | idb : ~0ull;
      }
    }
  } else
  for (int c = warp; c < n2; c += 8) {
    unsigned long long key = ~0ull;
    uint32_t id = c < C ? cid[c] : kInvalidId;
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
  if constexpr (kRefine) {
    // second stage: the first min(C, 2k) again, on both BF16 parts of each row
    const int m = min(C, 2 * k);
    const int m2 = pow2_at_least(m);
    const uint16_t* Xh = reinterpret_cast<const uint16_t*>(Xv);
    for (int c = warp; c < m2; c += 8) {
      unsigned long long key = ~0ull;
      const uint32_t id = c < m ? (uint32_t)(keys[c] & 0xFFFFFFFFu) : kInvalidId;
      if (c < m && keys[c] != ~0ull) {
        const uint16_t* xh = Xh + (size_t)id * d;
        const uint16_t* xl = Xl + (size_t)id * d;
        float acc = 0.f;
        for (int t = lane * 8; t < d; t += 256) {  // d % 8 == 0 in the precision form
          const uint4 vh = __ldg(reinterpret_cast<const uint4*>(xh + t));
          const uint4 vl = __ldg(reinterpret_cast<const uint4*>(xl + t));
          const uint32_t wh[4] = {vh.x, vh.y, vh.z, vh.w}, wl[4] = {vl.x, vl.y, vl.z, vl.w};
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const float x0 = __uint_as_float(wh[h] << 16) + __uint_as_float(wl[h] << 16);
            const float x1 = __uint_as_float(wh[h] & 0xFFFF0000u) + __uint_as_float(wl[h] & 0xFFFF0000u);
            const float a0 = sq[t + 2 * h] - x0, a1 = sq[t + 2 * h + 1] - x1;
            acc = fmaf(a0, a0, acc);
            acc = fmaf(a1, a1, acc);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        key = ((unsigned long long)__float_as_uint(acc) << 32) | id;
      }
      __syncwarp();
      // every warp reads its own entries only, so they can be replaced in place
      if (lane == 0) keys[c] = key;
    }
    __syncthreads();
    bitonic_sort_u64(keys, m2);
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    unsigned long long kk = i < n2 ? keys[i] : ~0ull;
    bool ok = kk != ~0ull;
    oid[i] = ok ? (int64_t)(kk & 0xFFFFFFFFu) : -1;
    od[i] = ok ? __uint_as_float((uint32_t)(kk >> 32)) : INFINITY;
  }
}

}  // namespace
}  // namespace hntl
