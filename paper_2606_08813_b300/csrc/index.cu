// Index file loader, Block-SoA device layout, index lifetime.
//
// The file is written by whoever built the index (the format is stated in
// include/hntl.h). Loading validates every size, offset and id and the
// trailing checksum, then re-lays the grain-ordered rows into 128-row blocks
// per grain (dimension-major inside a block, sec. 2.4's Block-SoA idea with
// the block sized for one GPU thread per row) and uploads them.
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hntl_internal.cuh"

namespace hntl {

static thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
void clear_error() { g_last_error.clear(); }

namespace {

constexpr char kMagic[8] = {'H', 'N', 'T', 'L', 'I', 'D', 'X', '\0'};
constexpr uint32_t kVersion = 1;
constexpr uint32_t kFlagEig = 1, kFlagFp8 = 2, kFlagXbf16 = 4, kFlagAttr = 8;
constexpr size_t kHeaderBytes = 40;

// Position-weighted word sum: sum over little-endian u64 words w_i (the last
// one zero padded) of w_i * (2 i + 1), modulo 2^64.
uint64_t word_sum(const uint8_t* p, size_t n) {
  uint64_t s = 0;
  size_t nw = n / 8;
  for (size_t i = 0; i < nw; ++i) {
    uint64_t w;
    std::memcpy(&w, p + 8 * i, 8);
    s += w * (2 * (uint64_t)i + 1);
  }
  if (n % 8) {
    uint64_t w = 0;
    std::memcpy(&w, p + 8 * nw, n % 8);
    s += w * (2 * (uint64_t)nw + 1);
  }
  return s;
}

struct Reader {
  const uint8_t* p;
  size_t n, off = 0;
  const uint8_t* take(size_t bytes) {
    if (bytes > n - off) return nullptr;
    const uint8_t* q = p + off;
    off += bytes;
    return q;
  }
};

template <typename T>
int dev_upload(Index& I, T** dst, const void* src, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) return fail(HNTL_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  I.allocations.push_back(p);
  I.device_bytes += bytes;
  if (src) {
    e = cudaMemcpy(p, src, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(HNTL_ECUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
  }
  *dst = static_cast<T*>(p);
  return HNTL_OK;
}

void free_all(Index& I) {
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(I.device);
  for (void* p : I.allocations) cudaFree(p);
  I.allocations.clear();
  if (prev >= 0) cudaSetDevice(prev);
}

}  // namespace

void int16_quantize(const float* Z, const float* rho, const std::vector<uint64_t>& goff, uint32_t r,
                    std::vector<float>& delta, std::vector<float>& dres, std::vector<int16_t>& codes,
                    std::vector<float>& rho_q) {
  const uint32_t G = (uint32_t)goff.size() - 1;
  const uint64_t N = goff[G];
  delta.assign(G, 1.0f);
  dres.assign(G, 1.0f);
  codes.assign(N * r, 0);
  rho_q.assign(N, 0.0f);
  for (uint32_t g = 0; g < G; ++g) {
    float m = 0.0f, mr = 0.0f;
    for (uint64_t p = goff[g]; p < goff[g + 1]; ++p) {
      for (uint32_t j = 0; j < r; ++j) m = std::max(m, std::fabs(Z[p * r + j]));
      mr = std::max(mr, rho[p]);
    }
    mr = std::max(mr, (m * m) * 0x1p-20f);  // no finer than FP32 resolves next to the coordinates' energy
    if (m > 0.0f) delta[g] = m / 16383.0f;
    if (mr > 0.0f) dres[g] = mr / 32767.0f;
    for (uint64_t p = goff[g]; p < goff[g + 1]; ++p) {
      for (uint32_t j = 0; j < r; ++j) {
        const float c = std::rint(Z[p * r + j] / delta[g]);
        codes[p * r + j] = (int16_t)std::max(-32767.0f, std::min(32767.0f, c));
      }
      rho_q[p] = std::max(0.0f, std::min(65535.0f, std::rint(rho[p] / dres[g]))) * dres[g];
    }
  }
}

std::vector<uint64_t> rows_by_first_coord(const float* Z, uint32_t r, const uint32_t* ids,
                                          const std::vector<uint64_t>& goff) {
  const uint32_t G = (uint32_t)goff.size() - 1;
  std::vector<uint64_t> order(goff[G]);
  for (uint64_t p = 0; p < goff[G]; ++p) order[p] = p;
  for (uint32_t g = 0; g < G; ++g)
    std::sort(order.begin() + (ptrdiff_t)goff[g], order.begin() + (ptrdiff_t)goff[g + 1],
              [&](uint64_t a, uint64_t b) {
                const float za = Z[a * r], zb = Z[b * r];
                return za < zb || (za == zb && ids[a] < ids[b]);
              });
  return order;
}

int load_from_memory(const uint8_t* buf, size_t size, int device, uint32_t precision, Index& I) {
  const bool no_raw = precision & HNTL_LOAD_NO_RAW;  // Mode A only: the raw rows stay on the host
  const bool rprune = precision & HNTL_INT16_RESID_PRUNE;
  precision &= ~(HNTL_LOAD_NO_RAW | HNTL_INT16_RESID_PRUNE);
  if (rprune && precision != HNTL_PREC_INT16)
    return fail(HNTL_EINVAL, "residual-saturation pruning applies to the 16-bit form only");
  if (size < kHeaderBytes + 8) return fail(HNTL_EFORMAT, "index file truncated (no header)");
  if (std::memcmp(buf, kMagic, 8) != 0) return fail(HNTL_EFORMAT, "bad magic (not an HNTL index file)");
  uint32_t version, flags, d, G, r, reserved;
  uint64_t N;
  std::memcpy(&version, buf + 8, 4);
  std::memcpy(&flags, buf + 12, 4);
  std::memcpy(&N, buf + 16, 8);
  std::memcpy(&d, buf + 24, 4);
  std::memcpy(&G, buf + 28, 4);
  std::memcpy(&r, buf + 32, 4);
  std::memcpy(&reserved, buf + 36, 4);
  if (version != kVersion) return fail(HNTL_EFORMAT, "unsupported index version " + std::to_string(version));
  if (flags & ~(kFlagEig | kFlagFp8 | kFlagXbf16 | kFlagAttr)) return fail(HNTL_EFORMAT, "unknown flag bits");
  if (d == 0 || G == 0 || r == 0 || r > d || N >= (1ull << 32) - 1)
    return fail(HNTL_EFORMAT, "bad sizes in header");
  if (r > (uint32_t)kMaxR) return fail(HNTL_EINVAL, "tangent dimension r > 64 is not supported");
  if (G > kMaxG) return fail(HNTL_EINVAL, "more than 8192 grains is not supported");
  if (precision != HNTL_PREC_FP32 && precision != HNTL_PREC_BF16_FP8 && precision != HNTL_PREC_INT16)
    return fail(HNTL_EINVAL, "bad precision");
  if (precision == HNTL_PREC_BF16_FP8 && d % 8)  // BF16 rows move in 16-byte pieces
    return fail(HNTL_EINVAL, "the precision form needs d to be a multiple of 8");
  bool xbf16 = flags & kFlagXbf16;
  if (precision != HNTL_PREC_BF16_FP8 && xbf16)
    return fail(HNTL_EINVAL, "file holds BF16 raw rows; load it as BF16_FP8");
  if (precision == HNTL_PREC_BF16_FP8 && !((flags & kFlagFp8) && xbf16))
    return fail(HNTL_EINVAL, "file has no FP8 coordinates / BF16 rows for the precision form");

  // exact expected size
  unsigned __int128 need = kHeaderBytes;
  need += (unsigned __int128)G * d * 4 + (unsigned __int128)G * r * d * 4;
  if (flags & kFlagEig) need += (unsigned __int128)G * d * 8;
  need += (unsigned __int128)(G + 1) * 8 + (unsigned __int128)N * 4 + (unsigned __int128)N * r * 4 + N * 4;
  if (flags & kFlagFp8) need += (unsigned __int128)N * r + (unsigned __int128)G * 4;
  need += (unsigned __int128)N * d * (xbf16 ? 2 : 4);
  if (flags & kFlagAttr) need += (unsigned __int128)N * 8;
  need += 8;
  if (need != (unsigned __int128)size)
    return fail(HNTL_EFORMAT, "index file size " + std::to_string(size) + " does not match its header (expected " +
                                  std::to_string((unsigned long long)need) + ")");
  uint64_t stored;
  std::memcpy(&stored, buf + size - 8, 8);
  if (word_sum(buf, size - 8) != stored) return fail(HNTL_EFORMAT, "index file checksum mismatch");

  Reader R{buf, size - 8, kHeaderBytes};
  const float* M = reinterpret_cast<const float*>(R.take((size_t)G * d * 4));
  const float* U = reinterpret_cast<const float*>(R.take((size_t)G * r * d * 4));
  if (flags & kFlagEig) R.take((size_t)G * d * 8);
  const uint8_t* off_raw = R.take((size_t)(G + 1) * 8);
  const uint8_t* ids_raw = R.take((size_t)N * 4);
  const float* Z = reinterpret_cast<const float*>(R.take((size_t)N * r * 4));
  const float* rho = reinterpret_cast<const float*>(R.take((size_t)N * 4));
  const uint8_t* Z8 = nullptr;
  const float* scale = nullptr;
  if (flags & kFlagFp8) {
    Z8 = R.take((size_t)N * r);
    scale = reinterpret_cast<const float*>(R.take((size_t)G * 4));
  }
  const uint8_t* Xraw = R.take((size_t)N * d * (xbf16 ? 2 : 4));
  const uint8_t* attr_raw = (flags & kFlagAttr) ? R.take((size_t)N * 8) : nullptr;

  std::vector<uint64_t> goff(G + 1);
  std::memcpy(goff.data(), off_raw, (G + 1) * 8);
  if (goff[0] != 0 || goff[G] != N) return fail(HNTL_EFORMAT, "grain offsets do not span the rows");
  for (uint32_t g = 0; g < G; ++g)
    if (goff[g + 1] < goff[g]) return fail(HNTL_EFORMAT, "grain offsets decrease");
  std::vector<uint32_t> ids(N);
  std::memcpy(ids.data(), ids_raw, N * 4);
  {
    std::vector<uint8_t> seen(N, 0);
    for (uint64_t i = 0; i < N; ++i) {
      if (ids[i] >= N || seen[ids[i]]) return fail(HNTL_EFORMAT, "grain-ordered ids are not a permutation");
      seen[ids[i]] = 1;
    }
  }
  std::vector<int64_t> attr;
  if (attr_raw) {
    attr.resize(N);
    std::memcpy(attr.data(), attr_raw, N * 8);
  }

  // Block-SoA re-layout on the host
  I.device = device;
  I.n = N;
  I.d = d;
  I.G = G;
  I.r = r;
  I.precision = precision;
  I.i16_resid_prune = rprune;
  I.rp = (uint32_t)padded_r((int)r, (int)precision);
  I.has_attr = attr_raw != nullptr;
  I.h_blk_off.assign(G + 1, 0);
  std::vector<uint32_t> grain_rows(G);
  std::vector<uint64_t> padded(G);
  uint64_t nb = 0;
  for (uint32_t g = 0; g < G; ++g) {
    uint64_t ng = goff[g + 1] - goff[g];
    grain_rows[g] = (uint32_t)ng;
    I.h_blk_off[g] = (uint32_t)nb;
    uint64_t b = (ng + kBlockRows - 1) / kBlockRows;
    padded[g] = b * kBlockRows;
    nb += b;
    I.max_grain_rows = std::max<uint64_t>(I.max_grain_rows, ng);
  }
  I.h_blk_off[G] = (uint32_t)nb;
  I.n_blocks = nb;
  std::vector<uint64_t> sorted = padded;
  std::sort(sorted.begin(), sorted.end(), std::greater<uint64_t>());
  I.h_top_padded_prefix.assign(G + 1, 0);
  for (uint32_t g = 0; g < G; ++g) I.h_top_padded_prefix[g + 1] = I.h_top_padded_prefix[g] + sorted[g];

  const size_t rows_pad = nb * kBlockRows;
  std::vector<uint32_t> blk_grain(nb);
  const int rp = (int)I.rp, V = coord_lane((int)precision);
  std::vector<float> Zb(precision == HNTL_PREC_FP32 ? rows_pad * rp : 0, 0.0f);
  std::vector<uint8_t> Z8b(precision == HNTL_PREC_BF16_FP8 ? rows_pad * rp : 0, 0);
  std::vector<int16_t> Z16b(precision == HNTL_PREC_INT16 ? rows_pad * rp : 0, 0);
  std::vector<float> rho_b(rows_pad, 0.0f);
  std::vector<float> delta, dres, rho16;
  std::vector<int16_t> codes16;
  if (precision == HNTL_PREC_INT16) int16_quantize(Z, rho, goff, r, delta, dres, codes16, rho16);
  std::vector<uint32_t> ids_b(rows_pad, kInvalidId);
  std::vector<int64_t> attr_b(I.has_attr ? rows_pad : 0, 0);
  // within a grain, rows go to blocks in order of their first coordinate, so a
  // block spans a short interval of it (the scan's interval bound)
  const std::vector<uint64_t> order = rows_by_first_coord(Z, r, ids.data(), goff);
  for (uint32_t g = 0; g < G; ++g) {
    for (uint32_t b = I.h_blk_off[g]; b < I.h_blk_off[g + 1]; ++b) blk_grain[b] = g;
    for (uint64_t i = 0; i < grain_rows[g]; ++i) {
      uint64_t p = order[goff[g] + i];
      uint64_t b = I.h_blk_off[g] + i / kBlockRows, t = i % kBlockRows;
      for (uint32_t j = 0; j < r; ++j) {
        if (precision == HNTL_PREC_FP32) {
          Zb[zoff(b, (int)j, (int)t, rp, V)] = Z[p * r + j];
        } else if (precision == HNTL_PREC_INT16) {
          Z16b[zoff(b, (int)j, (int)t, rp, V)] = codes16[p * r + j];
        } else {
          Z8b[zoff(b, (int)j, (int)t, rp, V)] = Z8[p * r + j];
        }
      }
      if (precision == HNTL_PREC_INT16)  // the residual on its grid, as the scan uses it
        rho_b[b * kBlockRows + t] = rho16[p];
      else
        rho_b[b * kBlockRows + t] = rho[p];
      ids_b[b * kBlockRows + t] = ids[p];
      if (I.has_attr) attr_b[b * kBlockRows + t] = attr[ids[p]];
    }
  }

  int prev = -1;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return fail(HNTL_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  int rc = HNTL_OK;
  do {
    if ((rc = dev_upload(I, &I.M, M, (size_t)G * d * 4))) break;
    if ((rc = dev_upload(I, &I.U, U, (size_t)G * r * d * 4))) break;
    if ((rc = dev_upload(I, &I.blk_off, I.h_blk_off.data(), (size_t)(G + 1) * 4))) break;
    if ((rc = dev_upload(I, &I.grain_rows, grain_rows.data(), (size_t)G * 4))) break;
    if ((rc = dev_upload(I, &I.blk_grain, blk_grain.data(), nb * 4))) break;
    if (precision == HNTL_PREC_FP32) {
      if ((rc = dev_upload(I, &I.Zb, Zb.data(), rows_pad * rp * 4))) break;
      if (!no_raw && (rc = dev_upload(I, &I.X, Xraw, (size_t)N * d * 4))) break;
    } else if (precision == HNTL_PREC_INT16) {
      if ((rc = dev_upload(I, &I.Z16b, Z16b.data(), rows_pad * rp * 2))) break;
      if ((rc = dev_upload(I, &I.scale, delta.data(), (size_t)G * 4))) break;
      if ((rc = dev_upload(I, &I.dres, dres.data(), (size_t)G * 4))) break;
      if (!no_raw && (rc = dev_upload(I, &I.X, Xraw, (size_t)N * d * 4))) break;
    } else {
      if ((rc = dev_upload(I, &I.Z8b, Z8b.data(), rows_pad * rp))) break;
      if ((rc = dev_upload(I, &I.scale, scale, (size_t)G * 4))) break;
      if (!no_raw && (rc = dev_upload(I, &I.Xh, Xraw, (size_t)N * d * 2))) break;
    }
    if ((rc = dev_upload(I, &I.rho, rho_b.data(), rows_pad * 4))) break;
    {
      std::vector<float> rmin(nb, INFINITY);
      for (uint32_t g = 0; g < G; ++g)
        for (uint64_t i = 0; i < grain_rows[g]; ++i) {
          const uint64_t b = I.h_blk_off[g] + i / kBlockRows;
          rmin[b] = std::min(rmin[b], rho_b[b * kBlockRows + i % kBlockRows]);
        }
      if ((rc = dev_upload(I, &I.blk_rho_min, rmin.data(), nb * 4))) break;
    }
    if ((rc = dev_upload(I, &I.ids, ids_b.data(), rows_pad * 4))) break;
    if (I.has_attr && (rc = dev_upload(I, &I.attr_b, attr_b.data(), rows_pad * 8))) break;
  } while (0);
  if (rc == HNTL_OK) rc = finalize_index(I);
  if (rc != HNTL_OK) free_all(I);
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}

void release(Index& I) { free_all(I); }

}  // namespace hntl

extern "C" {

const char* hntl_version(void) { return "hntl-b300 0.1 (sm_103a)"; }

const char* hntl_last_error(void) { return hntl::g_last_error.c_str(); }

int hntl_index_load(const char* path, int device, uint32_t precision, hntl_index** out) {
  hntl::clear_error();
  if (!path || !out) return hntl::fail(HNTL_EINVAL, "null argument");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return hntl::fail(HNTL_EIO, std::string("cannot open ") + path);
  std::vector<uint8_t> buf;
  if (std::fseek(f, 0, SEEK_END) != 0) {
    std::fclose(f);
    return hntl::fail(HNTL_EIO, "seek failed");
  }
  long sz = std::ftell(f);
  std::fseek(f, 0, SEEK_SET);
  if (sz < 0) {
    std::fclose(f);
    return hntl::fail(HNTL_EIO, "tell failed");
  }
  try {
    buf.resize((size_t)sz);
  } catch (...) {
    std::fclose(f);
    return hntl::fail(HNTL_ENOMEM, "host allocation for the index file failed");
  }
  size_t got = sz ? std::fread(buf.data(), 1, (size_t)sz, f) : 0;
  std::fclose(f);
  if (got != (size_t)sz) return hntl::fail(HNTL_EIO, "short read");
  hntl_index* h = nullptr;
  try {
    h = new hntl_index();
    int rc = hntl::load_from_memory(buf.data(), buf.size(), device, precision, h->I);
    if (rc != HNTL_OK) {
      delete h;
      return rc;
    }
  } catch (...) {
    delete h;
    return hntl::fail(HNTL_ENOMEM, "host allocation failed while loading");
  }
  *out = h;
  return HNTL_OK;
}

int hntl_int16_quantize_host(const float* Z, const float* rho, const uint64_t* goff, uint32_t G, uint32_t r,
                             float* delta, float* dres, int16_t* codes, float* rho_grid) {
  hntl::clear_error();
  if (!Z || !rho || !goff || !delta || !dres || !codes || !rho_grid) return hntl::fail(HNTL_EINVAL, "null argument");
  if (G == 0 || r == 0) return hntl::fail(HNTL_EINVAL, "G and r must be positive");
  if (goff[0] != 0) return hntl::fail(HNTL_EINVAL, "grain offsets must start at 0");
  for (uint32_t g = 0; g < G; ++g)
    if (goff[g + 1] < goff[g]) return hntl::fail(HNTL_EINVAL, "grain offsets decrease");
  try {
    const std::vector<uint64_t> off(goff, goff + G + 1);
    std::vector<float> dl, dr, rq;
    std::vector<int16_t> cq;
    hntl::int16_quantize(Z, rho, off, r, dl, dr, cq, rq);
    std::copy(dl.begin(), dl.end(), delta);
    std::copy(dr.begin(), dr.end(), dres);
    std::copy(cq.begin(), cq.end(), codes);
    std::copy(rq.begin(), rq.end(), rho_grid);
  } catch (...) {
    return hntl::fail(HNTL_ENOMEM, "host allocation failed");
  }
  return HNTL_OK;
}

int hntl_index_info(const hntl_index* idx, hntl_index_desc* out) {
  hntl::clear_error();
  if (!idx || !out) return hntl::fail(HNTL_EINVAL, "null argument");
  const hntl::Index& I = idx->I;
  out->n = I.n;
  out->d = I.d;
  out->G = I.G;
  out->r = I.r;
  out->precision = I.precision;
  out->has_attr = I.has_attr ? 1u : 0u;
  out->block_rows = hntl::kBlockRows;
  out->n_blocks = I.n_blocks;
  out->max_grain_rows = I.max_grain_rows;
  out->device_bytes = I.device_bytes;
  out->device = I.device;
  return HNTL_OK;
}

void hntl_index_free(hntl_index* idx) {
  if (!idx) return;
  hntl::release(idx->I);
  delete idx;
}

}  // extern "C"

// ------------------------------------------------------------------ export

namespace hntl {
namespace {

__global__ void k_export_rows(const uint32_t* __restrict__ blk_off, const uint32_t* __restrict__ grain_rows, int G,
                              int r, int rp, const float* __restrict__ Zb, const uint8_t* __restrict__ Z8b,
                              const int16_t* __restrict__ Z16b,
                              const float* __restrict__ scale, const float* __restrict__ rho_b,
                              const uint32_t* __restrict__ ids_b, const uint64_t* __restrict__ goff, float* __restrict__ Z,
                              float* __restrict__ rho, uint32_t* __restrict__ ids, uint64_t N) {
  uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  int lo = 0, hi = G;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (goff[mid] <= p) lo = mid;
    else hi = mid;
  }
  const int g = lo;
  const uint64_t i = p - goff[g];
  const size_t b = blk_off[g] + i / kBlockRows, t = i % kBlockRows;
  for (int j = 0; j < r; ++j) {
    float v;
    if (Zb) {
      v = Zb[zoff(b, j, (int)t, rp, 4)];
    } else if (Z16b) {
      v = (float)Z16b[zoff(b, j, (int)t, rp, 8)] * scale[g];
    } else {
      __nv_fp8_e4m3 c;
      c.__x = Z8b[zoff(b, j, (int)t, rp, 16)];
      v = (float)c * scale[g];
    }
    Z[p * r + j] = v;
  }
  rho[p] = rho_b[b * kBlockRows + t];
  ids[p] = ids_b[b * kBlockRows + t];
}

}  // namespace
}  // namespace hntl

extern "C" int hntl_index_grain_rows(const hntl_index* idx, uint32_t* h_rows) {
  hntl::clear_error();
  if (!idx || !h_rows) return hntl::fail(HNTL_EINVAL, "null argument");
  HNTL_CUDA_TRY(cudaMemcpy(h_rows, idx->I.grain_rows, sizeof(uint32_t) * idx->I.G, cudaMemcpyDeviceToHost));
  return HNTL_OK;
}

extern "C" int hntl_index_export(const hntl_index* idx, float* h_M, float* h_U, uint64_t* h_grain_off,
                                 uint32_t* h_ids, float* h_Z, float* h_rho) {
  hntl::clear_error();
  if (!idx) return hntl::fail(HNTL_EINVAL, "null index");
  const hntl::Index& I = idx->I;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(I.device);
  std::vector<uint32_t> rows(I.G);
  HNTL_CUDA_TRY(cudaMemcpy(rows.data(), I.grain_rows, sizeof(uint32_t) * I.G, cudaMemcpyDeviceToHost));
  std::vector<uint64_t> goff(I.G + 1, 0);
  for (uint32_t g = 0; g < I.G; ++g) goff[g + 1] = goff[g] + rows[g];
  if (h_grain_off) std::memcpy(h_grain_off, goff.data(), sizeof(uint64_t) * (I.G + 1));
  if (h_M) HNTL_CUDA_TRY(cudaMemcpy(h_M, I.M, sizeof(float) * I.G * I.d, cudaMemcpyDeviceToHost));
  if (h_U) HNTL_CUDA_TRY(cudaMemcpy(h_U, I.U, sizeof(float) * I.G * I.r * I.d, cudaMemcpyDeviceToHost));
  if (h_ids || h_Z || h_rho) {
    void *dZ = nullptr, *drho = nullptr, *dids = nullptr, *dgoff = nullptr;
    int rc = HNTL_OK;
    if (cudaMalloc(&dZ, std::max<size_t>(16, sizeof(float) * I.n * I.r)) != cudaSuccess ||
        cudaMalloc(&drho, std::max<size_t>(16, sizeof(float) * I.n)) != cudaSuccess ||
        cudaMalloc(&dids, std::max<size_t>(16, sizeof(uint32_t) * I.n)) != cudaSuccess ||
        cudaMalloc(&dgoff, sizeof(uint64_t) * (I.G + 1)) != cudaSuccess) {
      rc = hntl::fail(HNTL_ENOMEM, "export staging allocation failed");
    }
    if (rc == HNTL_OK) {
      cudaMemcpy(dgoff, goff.data(), sizeof(uint64_t) * (I.G + 1), cudaMemcpyHostToDevice);
      hntl::k_export_rows<<<(unsigned)((I.n + 255) / 256), 256>>>(
          I.blk_off, I.grain_rows, (int)I.G, (int)I.r, (int)I.rp, I.Zb, I.Z8b, I.Z16b, I.scale, I.rho, I.ids,
          static_cast<uint64_t*>(dgoff), static_cast<float*>(dZ), static_cast<float*>(drho),
          static_cast<uint32_t*>(dids), I.n);
      cudaError_t e = cudaDeviceSynchronize();
      if (e != cudaSuccess) rc = hntl::fail(HNTL_ECUDA, std::string("export: ") + cudaGetErrorString(e));
    }
    if (rc == HNTL_OK && h_Z) cudaMemcpy(h_Z, dZ, sizeof(float) * I.n * I.r, cudaMemcpyDeviceToHost);
    if (rc == HNTL_OK && h_rho) cudaMemcpy(h_rho, drho, sizeof(float) * I.n, cudaMemcpyDeviceToHost);
    if (rc == HNTL_OK && h_ids) cudaMemcpy(h_ids, dids, sizeof(uint32_t) * I.n, cudaMemcpyDeviceToHost);
    cudaFree(dZ);
    cudaFree(drho);
    cudaFree(dids);
    cudaFree(dgoff);
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
  }
  if (prev >= 0) cudaSetDevice(prev);
  return HNTL_OK;
}
