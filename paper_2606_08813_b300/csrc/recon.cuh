// Mode A of the query path (sec. 2.1 step 4, sec. 1): the pool reranked by
// the squared distance from the query to each row's reconstruction
// mu_g + W_g z_i (the subspace reconstruction of Eq. 3), with no raw row read.
//
// With v' = q - mu_g (the query as routed and projected) and z_q = U_g v',
//   ||v' - U_g^T z_i||^2 = ||v'||^2 - 2 z_i . z_q + z_i^T (U_g U_g^T) z_i
// for any basis U_g (the BF16 bases of the precision form are not exactly
// orthonormal). ||v'||^2 is the pair's exact routing distance, z_q its
// projection, and h_i = z_i^T G_g z_i is kept per row, so a pool member costs
// its position, its coordinates and two scalars instead of its d-value row.
#pragma once

#include "hntl_internal.cuh"
#include "kernels_common.cuh"
#include "scan_select.cuh"

namespace hntl {
namespace {

// Stored position (block * 128 + row) of every id; padding rows carry no id.
__global__ void k_pos_of_id(const uint32_t* __restrict__ ids, size_t npos, uint32_t* __restrict__ pos_of_id) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < npos && ids[i] != kInvalidId) pos_of_id[ids[i]] = (uint32_t)i;
}

// Per grain (FP32 form): U_g U_g^T (r x r, FP32 sums), one warp per entry.
__global__ void k_gram_f32(const float* __restrict__ U, int d, int r, float* __restrict__ gram) {
  const int g = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int e = warp; e < r * r; e += nw) {
    const int a = e / r, b = e % r;
    const float* ua = U + ((size_t)g * r + a) * d;
    const float* ub = U + ((size_t)g * r + b) * d;
    float acc = 0.f;
    for (int t = lane; t < d; t += 32) acc = fmaf(ua[t], ub[t], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) gram[((size_t)g * r + a) * r + b] = acc;
  }
}

// h_i = z_i^T G_g z_i of every stored row, z_i decoded exactly as the scan
// decodes it (padding rows get a harmless value that is never read).
template <int RT, int kC>
__global__ void __launch_bounds__(kBlockRows) k_row_h(const Coords cz, const uint32_t* __restrict__ blk_grain,
                                                      const float* __restrict__ gram, int r, int rp,
                                                      float* __restrict__ h_out) {
  const size_t b = blockIdx.x;
  const int t = threadIdx.x;
  const uint32_t g = blk_grain[b];
  float z[RT];
  load_row<RT, kC>(cz, rp, kC != kCoordF32 ? cz.scale[g] : 1.f, b, t, z);
  const float* Gg = gram + (size_t)g * r * r;
  float h = 0.f;
#pragma unroll
  for (int a = 0; a < RT; ++a) {
    if (a < r) {
      float acc = 0.f;
#pragma unroll
      for (int c = 0; c < RT; ++c)
        if (c < r) acc = fmaf(Gg[a * r + c], z[c], acc);
      h = fmaf(z[a], acc, h);
    }
  }
  h_out[b * kBlockRows + t] = h;
}

// One CTA per query: the reconstruction distance of every pool member (one
// thread each), then the k smallest (dist, id). A member's grain is one of
// the query's probes (the pool only holds rows of probed grains), which
// gives its (query, grain) pair: z_q and ||v'||^2.
template <int RT, int kC>
__global__ void __launch_bounds__(256) k_rerank_recon(int nprobe, int C, int k, const uint32_t* __restrict__ cand_id,
                                                      const uint32_t* __restrict__ pos_of_id,
                                                      const uint32_t* __restrict__ blk_grain, const Coords cz,
                                                      int r, int rp, const float* __restrict__ hrow,
                                                      const int32_t* __restrict__ probe,
                                                      const uint32_t* __restrict__ pair_of,
                                                      const float* __restrict__ zq,
                                                      const float* __restrict__ pair_vn,
                                                      int64_t* __restrict__ out_ids, float* __restrict__ out_d,
                                                      const uint32_t* __restrict__ qk,
                                                      const uint32_t* __restrict__ qC) {
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
  const int32_t* pq = probe + (size_t)q * nprobe;
  const uint32_t* po = pair_of + (size_t)q * nprobe;
  const int n2 = pow2_at_least(C);
  for (int c = threadIdx.x; c < n2; c += blockDim.x) {
    unsigned long long key = ~0ull;
    const uint32_t id = c < C ? cid[c] : kInvalidId;
    if (id != kInvalidId) {
      const uint32_t pos = pos_of_id[id];
      const size_t b = pos / kBlockRows;
      const int t = (int)(pos % kBlockRows);
      const uint32_t g = blk_grain[b];
      int p = 0;
      while (p + 1 < nprobe && (uint32_t)pq[p] != g) ++p;
      const uint32_t pr = po[p];
      float z[RT];
      load_row<RT, kC>(cz, rp, kC != kCoordF32 ? cz.scale[g] : 1.f, b, t, z);
      const float* zp = zq + (size_t)pr * r;
      float dot = 0.f;
#pragma unroll
      for (int a = 0; a < RT; ++a)
        if (a < r) dot = fmaf(z[a], zp[a], dot);
      const float dA = fmaxf((pair_vn[pr] - 2.f * dot) + hrow[pos], 0.f);  // >= 0 up to rounding
      key = ((unsigned long long)__float_as_uint(dA) << 32) | id;
    }
    keys[c] = key;
  }
  __syncthreads();
  bitonic_sort_u64(keys, n2);
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const unsigned long long kk = i < n2 ? keys[i] : ~0ull;
    const bool ok = kk != ~0ull;
    oid[i] = ok ? (int64_t)(kk & 0xFFFFFFFFu) : -1;
    od[i] = ok ? __uint_as_float((uint32_t)(kk >> 32)) : INFINITY;
  }
}

}  // namespace
}  // namespace hntl
