// Grain shards of an index, and the merge of the shards' results.
//
// The query path splits over devices by grains (sec. 2.1 steps 1-4 run per
// grain, and a query's answer is the best k over the grains it probes):
// every shard keeps all G centres and bases, so it routes each query exactly
// as the whole index does, but holds the rows, coordinates and raw rows of
// its own grains only (the other grains are empty). Each shard scans its
// probed grains, keeps its own pool of C and reranks it to its own top k; the
// merge then takes the k best by (distance, id) over all shards' lists. The
// union of the shards' pools contains the whole index's pool, so the merged
// top k is the exact-distance top k of a superset of the single-index pool.
//
// A shard numbers its rows 0..n_s-1 in ascending original id, so that equal
// distances break ties in the same order as in the whole index, and keeps
// the original id of each row (gid) to map its results back.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "hntl_internal.cuh"

namespace hntl {
namespace {

__global__ void k_gather_rows(const uint16_t* __restrict__ src, const uint32_t* __restrict__ gid, uint64_t n,
                              uint32_t units, uint16_t* __restrict__ dst) {
  // rows of `units` 16-bit units (BF16 rows: d; FP32 rows: 2 d)
  const uint64_t total = n * units;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t row = e / units, u = e - row * units;
    dst[e] = src[(uint64_t)gid[row] * units + u];
  }
}

__global__ void k_global_ids(int64_t* __restrict__ ids, uint64_t n, const uint32_t* __restrict__ gid, uint64_t n_s) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const int64_t v = ids[i];
    ids[i] = (v >= 0 && (uint64_t)v < n_s) ? (int64_t)gid[v] : -1;
  }
}

// (distance, id) order of the merge; an id < 0 (padding) ranks after every real entry
__host__ __device__ inline bool merge_less(float da, int64_t ia, float db, int64_t ib) {
  const bool va = ia >= 0, vb = ib >= 0;
  if (va != vb) return va;
  if (!va) return false;
  if (da != db) return da < db;
  return ia < ib;
}

// One warp per query: k rounds, each taking the smallest (distance, id) above
// the previous round's over the S k candidates (ids are distinct across shards).
__global__ void k_merge_topk(const int64_t* __restrict__ ids, const float* __restrict__ dist, uint32_t S,
                             uint32_t nq, uint32_t k, int64_t* __restrict__ out_ids, float* __restrict__ out_d) {
  const uint32_t q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= nq) return;
  const uint32_t m = S * k;
  float pd = -INFINITY;
  int64_t pi = INT64_MIN;
  bool have_prev = false;
  for (uint32_t t = 0; t < k; ++t) {
    float bd = INFINITY;
    int64_t bi = -1;
    for (uint32_t c = lane; c < m; c += 32) {
      const uint32_t s = c / k, j = c - s * k;
      const size_t at = ((size_t)s * nq + q) * k + j;
      const int64_t i = ids[at];
      const float dd = dist[at];
      if (i < 0) continue;
      if (have_prev && !merge_less(pd, pi, dd, i)) continue;  // taken in an earlier round
      if (merge_less(dd, i, bd, bi)) {
        bd = dd;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float od = __shfl_xor_sync(0xffffffffu, bd, o);
      const long long oi = __shfl_xor_sync(0xffffffffu, (long long)bi, o);
      if (merge_less(od, oi, bd, bi)) {
        bd = od;
        bi = oi;
      }
    }
    if (lane == 0) {
      out_ids[(size_t)q * k + t] = bi;
      out_d[(size_t)q * k + t] = bi >= 0 ? bd : INFINITY;
    }
    if (bi < 0) {  // fewer than k real entries: pad the rest
      for (uint32_t u = t + 1 + lane; u < k; u += 32) {
        out_ids[(size_t)q * k + u] = -1;
        out_d[(size_t)q * k + u] = INFINITY;
      }
      break;
    }
    pd = bd;
    pi = bi;
    have_prev = true;
  }
}

template <typename T>
int upload(Index& I, T** dst, const void* src, size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) return fail(HNTL_ENOMEM, "shard: device allocation");
  I.allocations.push_back(p);
  I.device_bytes += std::max<size_t>(bytes, 16);
  if (src && bytes) HNTL_CUDA_TRY(cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice));
  *dst = static_cast<T*>(p);
  return HNTL_OK;
}

// Copy blocks [b0, b1) of a per-block device array (`per` elements of T a block) to host.
template <typename T>
int fetch_blocks(const T* src, uint64_t b0, uint64_t b1, size_t per, std::vector<T>& dst) {
  const size_t at = dst.size();
  dst.resize(at + (b1 - b0) * per);
  if (b1 > b0) HNTL_CUDA_TRY(cudaMemcpy(dst.data() + at, src + b0 * per, (b1 - b0) * per * sizeof(T), cudaMemcpyDeviceToHost));
  return HNTL_OK;
}

int make_shard(const Index& S, const uint32_t* shard_of, uint32_t shard, int device, Index& I) {
  const uint32_t G = S.G, d = S.d, r = S.r, rp = S.rp;
  std::vector<uint32_t> rows(G);
  HNTL_CUDA_TRY(cudaSetDevice(S.device));
  HNTL_CUDA_TRY(cudaMemcpy(rows.data(), S.grain_rows, sizeof(uint32_t) * G, cudaMemcpyDeviceToHost));
  std::vector<float> M((size_t)G * d), U((size_t)G * r * d), scale, dres;
  HNTL_CUDA_TRY(cudaMemcpy(M.data(), S.M, M.size() * 4, cudaMemcpyDeviceToHost));
  HNTL_CUDA_TRY(cudaMemcpy(U.data(), S.U, U.size() * 4, cudaMemcpyDeviceToHost));
  if (S.scale) {
    scale.resize(G);
    HNTL_CUDA_TRY(cudaMemcpy(scale.data(), S.scale, G * 4, cudaMemcpyDeviceToHost));
  }
  if (S.dres) {
    dres.resize(G);
    HNTL_CUDA_TRY(cudaMemcpy(dres.data(), S.dres, G * 4, cudaMemcpyDeviceToHost));
  }
  // the shard's blocks: every block of each owned grain, in grain order
  std::vector<uint32_t> blk_off(G + 1, 0), grain_rows(G, 0);
  std::vector<uint32_t> ids;
  std::vector<float> rho, rmin, Zb;
  std::vector<uint8_t> Z8b;
  std::vector<int16_t> Z16b;
  std::vector<int64_t> attr;
  const size_t cpb = (size_t)rp * kBlockRows;  // coordinates per block
  uint64_t nb = 0, max_rows = 0;
  for (uint32_t g = 0; g < G; ++g) {
    blk_off[g] = (uint32_t)nb;
    if (shard_of[g] != shard) continue;
    const uint64_t b0 = S.h_blk_off[g], b1 = S.h_blk_off[g + 1];
    grain_rows[g] = rows[g];
    max_rows = std::max<uint64_t>(max_rows, rows[g]);
    nb += b1 - b0;
    int rc;
    if ((rc = fetch_blocks(S.ids, b0, b1, kBlockRows, ids)) || (rc = fetch_blocks(S.rho, b0, b1, kBlockRows, rho)) ||
        (rc = fetch_blocks(S.blk_rho_min, b0, b1, 1, rmin)))
      return rc;
    if (S.Zb && (rc = fetch_blocks(S.Zb, b0, b1, cpb, Zb))) return rc;
    if (S.Z8b && (rc = fetch_blocks(S.Z8b, b0, b1, cpb, Z8b))) return rc;
    if (S.Z16b && (rc = fetch_blocks(S.Z16b, b0, b1, cpb, Z16b))) return rc;
    if (S.has_attr && (rc = fetch_blocks(S.attr_b, b0, b1, kBlockRows, attr))) return rc;
  }
  blk_off[G] = (uint32_t)nb;
  // local ids: the shard's rows in ascending original id
  std::vector<uint32_t> gid;
  gid.reserve(ids.size());
  for (uint32_t v : ids)
    if (v != kInvalidId) gid.push_back(v);
  std::sort(gid.begin(), gid.end());
  for (uint32_t& v : ids)
    if (v != kInvalidId) v = (uint32_t)(std::lower_bound(gid.begin(), gid.end(), v) - gid.begin());
  const uint64_t n_s = gid.size();
  // raw rows of the shard (and their second BF16 parts), gathered on the source device
  const bool has_raw = S.X || S.Xh;
  const uint32_t units = S.Xh ? d : 2 * d;  // 16-bit units per raw row
  auto gather = [&](const uint16_t* src, std::vector<uint16_t>& out) -> int {
    out.assign(n_s * units, 0);
    if (!n_s) return HNTL_OK;
    const uint64_t chunk = std::min<uint64_t>(n_s, 1u << 20);
    uint32_t* dgid = nullptr;
    uint16_t* dtmp = nullptr;
    if (cudaMalloc(&dgid, n_s * 4) != cudaSuccess) return fail(HNTL_ENOMEM, "shard: staging");
    if (cudaMalloc(&dtmp, chunk * units * 2) != cudaSuccess) {
      cudaFree(dgid);
      return fail(HNTL_ENOMEM, "shard: staging");
    }
    cudaError_t e = cudaMemcpy(dgid, gid.data(), n_s * 4, cudaMemcpyHostToDevice);
    for (uint64_t a = 0; a < n_s && e == cudaSuccess; a += chunk) {
      const uint64_t m = std::min<uint64_t>(chunk, n_s - a);
      const uint64_t blocks = std::min<uint64_t>((m * units + 255) / 256, 65535);
      k_gather_rows<<<(unsigned)blocks, 256>>>(src, dgid + a, m, units, dtmp);
      e = cudaMemcpy(out.data() + a * units, dtmp, m * units * 2, cudaMemcpyDeviceToHost);
    }
    cudaFree(dgid);
    cudaFree(dtmp);
    if (e != cudaSuccess) return fail(HNTL_ECUDA, std::string("shard: raw rows: ") + cudaGetErrorString(e));
    return HNTL_OK;
  };
  std::vector<uint16_t> Xs, Xls;
  if (has_raw) {
    const int rc0 = gather(S.Xh ? S.Xh : reinterpret_cast<const uint16_t*>(S.X), Xs);
    if (rc0) return rc0;
  }
  if (S.Xl) {
    const int rc0 = gather(S.Xl, Xls);
    if (rc0) return rc0;
  }

  I.device = device;
  I.n = n_s;
  I.d = d;
  I.G = G;
  I.r = r;
  I.precision = S.precision;
  I.rp = rp;
  I.has_attr = S.has_attr;
  I.i16_resid_prune = S.i16_resid_prune;
  I.n_blocks = nb;
  I.max_grain_rows = max_rows;
  I.h_blk_off = blk_off;
  std::vector<uint64_t> padded(G);
  for (uint32_t g = 0; g < G; ++g) padded[g] = (uint64_t)(blk_off[g + 1] - blk_off[g]) * kBlockRows;
  std::sort(padded.begin(), padded.end(), std::greater<uint64_t>());
  I.h_top_padded_prefix.assign(G + 1, 0);
  for (uint32_t g = 0; g < G; ++g) I.h_top_padded_prefix[g + 1] = I.h_top_padded_prefix[g] + padded[g];
  std::vector<uint32_t> blk_grain(nb);
  for (uint32_t g = 0; g < G; ++g)
    for (uint32_t b = blk_off[g]; b < blk_off[g + 1]; ++b) blk_grain[b] = g;

  HNTL_CUDA_TRY(cudaSetDevice(device));
  int rc;
  if ((rc = upload(I, &I.M, M.data(), M.size() * 4)) || (rc = upload(I, &I.U, U.data(), U.size() * 4)) ||
      (rc = upload(I, &I.blk_off, blk_off.data(), (G + 1) * 4)) ||
      (rc = upload(I, &I.grain_rows, grain_rows.data(), G * 4)) ||
      (rc = upload(I, &I.blk_grain, blk_grain.data(), nb * 4)) ||
      (rc = upload(I, &I.rho, rho.data(), rho.size() * 4)) ||
      (rc = upload(I, &I.blk_rho_min, rmin.data(), rmin.size() * 4)) ||
      (rc = upload(I, &I.ids, ids.data(), ids.size() * 4)) || (rc = upload(I, &I.gid, gid.data(), n_s * 4)))
    return rc;
  if (S.Zb && (rc = upload(I, &I.Zb, Zb.data(), Zb.size() * 4))) return rc;
  if (S.Z8b && (rc = upload(I, &I.Z8b, Z8b.data(), Z8b.size()))) return rc;
  if (S.Z16b && (rc = upload(I, &I.Z16b, Z16b.data(), Z16b.size() * 2))) return rc;
  if (S.scale && (rc = upload(I, &I.scale, scale.data(), G * 4))) return rc;
  if (S.dres && (rc = upload(I, &I.dres, dres.data(), G * 4))) return rc;
  if (S.has_attr && (rc = upload(I, &I.attr_b, attr.data(), attr.size() * 8))) return rc;
  if (S.Xh && (rc = upload(I, &I.Xh, Xs.data(), Xs.size() * 2))) return rc;
  if (S.Xl && (rc = upload(I, &I.Xl, Xls.data(), Xls.size() * 2))) return rc;
  if (S.X && (rc = upload(I, &I.X, Xs.data(), Xs.size() * 2))) return rc;
  return finalize_index(I);
}

}  // namespace
}  // namespace hntl

extern "C" {

int hntl_shard_assign(const uint32_t* h_grain_rows, uint32_t G, uint32_t S, uint32_t* h_shard_of_grain) {
  hntl::clear_error();
  if (!h_grain_rows || !h_shard_of_grain || G == 0 || S == 0 || S > G) return hntl::fail(HNTL_EINVAL, "shard_assign: bad arguments");
  std::vector<uint32_t> order(G);
  std::iota(order.begin(), order.end(), 0u);
  std::stable_sort(order.begin(), order.end(),
                   [&](uint32_t a, uint32_t b) { return h_grain_rows[a] > h_grain_rows[b]; });
  std::vector<uint64_t> load(S, 0);
  for (uint32_t g : order) {
    uint32_t best = 0;
    for (uint32_t s = 1; s < S; ++s)
      if (load[s] < load[best]) best = s;
    h_shard_of_grain[g] = best;
    load[best] += h_grain_rows[g];
  }
  return HNTL_OK;
}

int hntl_index_shard(const hntl_index* idx, const uint32_t* h_shard_of_grain, uint32_t shard, int device,
                     hntl_index** out) {
  hntl::clear_error();
  if (!idx || !h_shard_of_grain || !out) return hntl::fail(HNTL_EINVAL, "null argument");
  *out = nullptr;
  const hntl::Index& S = idx->I;
  if (S.gid) return hntl::fail(HNTL_EINVAL, "index_shard: the index is itself a shard");
  bool any = false;
  for (uint32_t g = 0; g < S.G; ++g) any |= h_shard_of_grain[g] == shard;
  if (!any) return hntl::fail(HNTL_EINVAL, "index_shard: the shard owns no grain");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return hntl::fail(HNTL_EINVAL, "index_shard: bad device");
  int prev = -1;
  cudaGetDevice(&prev);
  hntl_index* h = new hntl_index();
  int rc = hntl::make_shard(S, h_shard_of_grain, shard, device, h->I);
  if (rc != HNTL_OK) {
    hntl::release(h->I);
    delete h;
  } else {
    *out = h;
  }
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}

int hntl_shard_global_ids(const hntl_index* shard, int64_t* d_ids, uint64_t count, void* stream) {
  hntl::clear_error();
  if (!shard || (!d_ids && count)) return hntl::fail(HNTL_EINVAL, "null argument");
  const hntl::Index& I = shard->I;
  if (!I.gid) return hntl::fail(HNTL_EINVAL, "shard_global_ids: the index is not a shard");
  if (count == 0) return HNTL_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(I.device);
  hntl::k_global_ids<<<(unsigned)((count + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(d_ids, count,
                                                                                                     I.gid, I.n);
  cudaError_t e = cudaGetLastError();
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess) return hntl::fail(HNTL_ECUDA, std::string("shard_global_ids: ") + cudaGetErrorString(e));
  return HNTL_OK;
}

int hntl_merge_topk(const int64_t* d_ids, const float* d_dist, uint32_t S, uint32_t nq, uint32_t k,
                    int64_t* d_out_ids, float* d_out_dist, void* stream) {
  hntl::clear_error();
  if (S == 0 || k == 0 || (nq && (!d_ids || !d_dist || !d_out_ids || !d_out_dist)))
    return hntl::fail(HNTL_EINVAL, "merge_topk: bad arguments");
  if ((uint64_t)S * k > (1u << 24)) return hntl::fail(HNTL_EINVAL, "merge_topk: S k too large");
  if (nq == 0) return HNTL_OK;
  hntl::k_merge_topk<<<(nq + 7) / 8, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_ids, d_dist, S, nq, k, d_out_ids,
                                                                                  d_out_dist);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return hntl::fail(HNTL_ECUDA, std::string("merge_topk: ") + cudaGetErrorString(e));
  return HNTL_OK;
}

int hntl_merge_topk_host(const int64_t* h_ids, const float* h_dist, uint32_t S, uint32_t nq, uint32_t k,
                         int64_t* h_out_ids, float* h_out_dist) {
  hntl::clear_error();
  if (S == 0 || k == 0 || (nq && (!h_ids || !h_dist || !h_out_ids || !h_out_dist)))
    return hntl::fail(HNTL_EINVAL, "merge_topk_host: bad arguments");
  std::vector<std::pair<float, int64_t>> c;
  for (uint32_t q = 0; q < nq; ++q) {
    c.clear();
    for (uint32_t s = 0; s < S; ++s)
      for (uint32_t j = 0; j < k; ++j) {
        const size_t at = ((size_t)s * nq + q) * k + j;
        if (h_ids[at] >= 0) c.emplace_back(h_dist[at], h_ids[at]);
      }
    const size_t m = std::min<size_t>(k, c.size());
    std::partial_sort(c.begin(), c.begin() + m, c.end(), [](const auto& a, const auto& b) {
      return hntl::merge_less(a.first, a.second, b.first, b.second);
    });
    for (uint32_t j = 0; j < k; ++j) {
      h_out_ids[(size_t)q * k + j] = j < m ? c[j].second : -1;
      h_out_dist[(size_t)q * k + j] = j < m ? c[j].first : INFINITY;
    }
  }
  return HNTL_OK;
}

}  // extern "C"
