// Learned grain router: an MLP d -> h1 -> h2 -> G (exact GELU, softmax over
// grains) trained on the GPU with BF16 matrix products (tcgen05, FP32
// accumulation) and FP32 AdamW master weights, and used to choose each
// query's probed grains, with centroid routing as the fallback.
//
// Where values are rounded to BF16 (the only roundings besides FP32
// arithmetic):
//   forward:  X_b, W_b for each layer; H1_b = bf16(gelu(A1)); H2_b = bf16(gelu(A2))
//   backward: dL_b = bf16((P - T) / B); dA2_b = bf16(dH2 * gelu'(A2)); dA1_b = bf16(dH1 * gelu'(A1))
//   gradients: dW3 = dL_b^T H2_b, dW2 = dA2_b^T H1_b, dW1 = dA1_b^T X_b; bias gradients are
//              FP32 column sums of dL, dA2, dA1.
// The paper names learned grain partitioning as future work (sec. 4); the
// router itself, its labels (the grains holding a query's brute-force top 10,
// as soft targets) and its loss are this library's additions.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "gemm_tc.cuh"
#include "hntl_internal.cuh"
#include "route_kernels.cuh"

namespace hntl {

namespace {

__global__ void k_f32_to_bf16(const float* __restrict__ x, size_t n, uint16_t* __restrict__ y) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __bfloat16_as_ushort(__float2bfloat16_rn(x[i]));
}

// dst[c][r] = src[r][c] for a BF16 matrix [R][Cn], 32 x 32 tiles through shared memory.
__global__ void k_transpose_bf16(const uint16_t* __restrict__ src, int R, int Cn, uint16_t* __restrict__ dst) {
  __shared__ uint16_t tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < R && c < Cn) ? src[(size_t)r * Cn + c] : 0;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < Cn && r < R) dst[(size_t)c * R + r] = tile[threadIdx.x][i];
  }
}

__device__ float block_reduce(float v, float* red, bool is_max) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float u = __shfl_xor_sync(0xffffffffu, v, o);
    v = is_max ? fmaxf(v, u) : v + u;
  }
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float r = red[0];
  for (int i = 1; i < nw; ++i) r = is_max ? fmaxf(r, red[i]) : r + red[i];
  return r;
}

// One CTA per row: P = softmax(L), loss_i = -sum T log P, dL = (P - T) / B (FP32 and BF16).
__global__ void k_softmax_ce(const float* __restrict__ L, const float* __restrict__ T, int G, int B,
                             float* __restrict__ dL, uint16_t* __restrict__ dLb, float* __restrict__ loss) {
  __shared__ float red[32];
  const int i = blockIdx.x;
  const float* l = L + (size_t)i * G;
  const float* t = T + (size_t)i * G;
  float m = -INFINITY;
  for (int g = threadIdx.x; g < G; g += blockDim.x) m = fmaxf(m, l[g]);
  m = block_reduce(m, red, true);
  float s = 0.f;
  for (int g = threadIdx.x; g < G; g += blockDim.x) s += expf(l[g] - m);
  s = block_reduce(s, red, false);
  const float ls = logf(s);
  float li = 0.f;
  for (int g = threadIdx.x; g < G; g += blockDim.x) {
    const float lp = l[g] - m - ls;  // log P
    const float p = expf(lp);
    if (t[g] > 0.f) li -= t[g] * lp;
    const float v = (p - t[g]) / (float)B;
    dL[(size_t)i * G + g] = v;
    dLb[(size_t)i * G + g] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
  }
  li = block_reduce(li, red, false);
  if (threadIdx.x == 0 && loss) atomicAdd(loss, li / (float)B);
}

// dA = dH * gelu'(A) (FP32 and BF16)
__global__ void k_gelu_bwd(const float* __restrict__ dH, const float* __restrict__ A, size_t n,
                           float* __restrict__ dA, uint16_t* __restrict__ dAb) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = dH[i] * gelu_grad_f(A[i]);
  dA[i] = v;
  dAb[i] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// out[c] = sum over rows of x[r][c] (the bias gradients). A block per 32
// columns, blockDim (32, kColGroups): thread (c, j) sums rows j, j + kColGroups,
// ... of its column (a warp reads 128 contiguous bytes of a row), then the
// group sums are added in group order, so the result does not depend on
// scheduling. One thread per column with a serial walk over the rows left
// most SMs idle and each thread latency-bound.
constexpr int kColGroups = 32;
__global__ void __launch_bounds__(32 * kColGroups) k_colsum(const float* __restrict__ x, int R, int Cn,
                                                            float* __restrict__ out) {
  __shared__ float part[kColGroups][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  float s = 0.f;
  if (c < Cn) {
#pragma unroll 8
    for (int r = threadIdx.y; r < R; r += kColGroups) s += x[(size_t)r * Cn + c];
  }
  part[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && c < Cn) {
    float t = 0.f;
#pragma unroll
    for (int j = 0; j < kColGroups; ++j) t += part[j][threadIdx.x];
    out[c] = t;
  }
}

// Advances the AdamW step count and stores its bias corrections.
__global__ void k_adam_tick(unsigned long long* step, float* bc, float b1, float b2) {
  const unsigned long long t = ++*step;
  bc[0] = 1.f - powf(b1, (float)t);
  bc[1] = 1.f - powf(b2, (float)t);
}

// The six parameter tensors of one AdamW update; block b works on tensor i
// where blk[i] <= b < blk[i + 1].
struct AdamSet {
  float* p[6];
  const float* g[6];
  float* m[6];
  float* v[6];
  uint16_t* pb[6];  // BF16 copy to refresh, or nullptr
  size_t n[6];
  float wd[6];
  unsigned blk[7];
};

// Decoupled weight decay Adam on FP32 masters (all six tensors in one
// launch); refreshes the BF16 copies.
__global__ void k_adamw(const AdamSet S, float lr, float b1, float b2, float eps, const float* __restrict__ bc) {
  int i = 0;
  while (i < 5 && blockIdx.x >= S.blk[i + 1]) ++i;
  const size_t j = (size_t)(blockIdx.x - S.blk[i]) * blockDim.x + threadIdx.x;
  if (j >= S.n[i]) return;
  const float c1 = bc[0], c2 = bc[1];
  const float gi = S.g[i][j];
  const float mi = b1 * S.m[i][j] + (1.f - b1) * gi;
  const float vi = b2 * S.v[i][j] + (1.f - b2) * gi * gi;
  S.m[i][j] = mi;
  S.v[i][j] = vi;
  const float p = S.p[i][j];
  const float w = p - lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + S.wd[i] * p);
  S.p[i][j] = w;
  if (S.pb[i]) S.pb[i][j] = __bfloat16_as_ushort(__float2bfloat16_rn(w));
}

// Per row: m = max logit, s = sum exp(l - m); writes -l (so the routing select's ascending order picks the
// largest logits).
__global__ void k_logit_stats(const float* __restrict__ L, int G, float* __restrict__ negl, float* __restrict__ mx,
                              float* __restrict__ sm) {
  __shared__ float red[32];
  const int i = blockIdx.x;
  const float* l = L + (size_t)i * G;
  float m = -INFINITY;
  for (int g = threadIdx.x; g < G; g += blockDim.x) m = fmaxf(m, l[g]);
  m = block_reduce(m, red, true);
  float s = 0.f;
  for (int g = threadIdx.x; g < G; g += blockDim.x) {
    s += expf(l[g] - m);
    negl[(size_t)i * G + g] = -l[g];
  }
  s = block_reduce(s, red, false);
  if (threadIdx.x == 0) {
    mx[i] = m;
    sm[i] = s;
  }
}

// Keep the router's probes where their softmax mass reaches tau; otherwise take the centroid probes.
__global__ void k_router_merge(int nq, int nprobe, const float* __restrict__ neg_top, const float* __restrict__ mx,
                               const float* __restrict__ sm, float tau, const int32_t* __restrict__ centroid_probe,
                               int32_t* __restrict__ probe, uint32_t* __restrict__ nfallback) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  float mass = 0.f;
  for (int p = 0; p < nprobe; ++p) mass += expf(-neg_top[(size_t)q * nprobe + p] - mx[q]);
  mass /= sm[q];
  if (!(mass >= tau)) {
    for (int p = 0; p < nprobe; ++p) probe[(size_t)q * nprobe + p] = centroid_probe[(size_t)q * nprobe + p];
    if (nfallback) atomicAdd(nfallback, 1u);
  }
}

// The fused selection below handles up to this many probes and 256 x 32 grains.
constexpr int kTopMax = 64;

// One CTA of 256 threads per query, straight from its G logits: the max and
// the sum of exp(l - max) in the same per-thread order and block reduction as
// k_logit_stats (so both are bitwise the same), the nprobe largest logits
// (ties to the lower grain, NaN last) by nprobe rounds of a block-wide minimum
// over (negated logit, grain) keys held in registers, their softmax mass
// summed in selection order as k_router_merge does, and the probes: the
// centroid probes where that mass is below tau (centroid_probe null: no query
// falls back).
template <int kPer>
__global__ void __launch_bounds__(256) k_router_topk(const float* __restrict__ L, int G, int nprobe, float tau,
                                                     const int32_t* __restrict__ centroid_probe,
                                                     int32_t* __restrict__ probe, uint32_t* __restrict__ nfallback) {
  __shared__ float red[32];
  __shared__ unsigned long long wmin[8];
  __shared__ unsigned long long pick[kTopMax];
  __shared__ int s_fall;
  const int q = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const float* l = L + (size_t)q * G;
  float v[kPer];
  float m = -INFINITY;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int g = t + 256 * j;
    v[j] = g < G ? l[g] : -INFINITY;
    m = fmaxf(m, v[j]);
  }
  m = block_reduce(m, red, true);
  float sum = 0.f;
#pragma unroll
  for (int j = 0; j < kPer; ++j)
    if (t + 256 * j < G) sum += expf(v[j] - m);
  sum = block_reduce(sum, red, false);
  unsigned long long key[kPer];
  unsigned long long lm = ~0ull;  // this thread's smallest key left
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int g = t + 256 * j;
    float x = -v[j];
    if (!(x == x)) x = INFINITY;  // a NaN logit ranks last
    if (x == 0.f) x = 0.f;        // -0 and +0 rank alike (ties go to the lower grain)
    const uint32_t b = __float_as_uint(x);
    const uint32_t hi = (b & 0x80000000u) ? ~b : (b | 0x80000000u);  // order-preserving
    key[j] = g < G ? ((unsigned long long)hi << 32) | (uint32_t)g : ~0ull;
    lm = min(lm, key[j]);
  }
  for (int p = 0; p < nprobe; ++p) {
    unsigned long long w = lm;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w = min(w, __shfl_xor_sync(0xffffffffu, w, o));
    if (lane == 0) wmin[warp] = w;
    __syncthreads();
    if (warp == 0) {
      unsigned long long x = lane < 8 ? wmin[lane] : ~0ull;
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
      if (lane == 0) pick[p] = x;
    }
    __syncthreads();
    const unsigned long long pk = pick[p];
    if (lm == pk) {  // keys are distinct: one thread owns it
      lm = ~0ull;
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        if (key[j] == pk) key[j] = ~0ull;
        lm = min(lm, key[j]);
      }
    }
  }
  if (t == 0) {
    float mass = 0.f;
    for (int p = 0; p < nprobe; ++p) {
      const uint32_t hi = (uint32_t)(pick[p] >> 32);
      const float x = __uint_as_float((hi & 0x80000000u) ? (hi & 0x7FFFFFFFu) : ~hi);  // the negated logit
      mass += expf(-x - m);
    }
    mass /= sum;
    const bool fall = centroid_probe != nullptr && !(mass >= tau);
    s_fall = fall;
    if (fall && nfallback) atomicAdd(nfallback, 1u);
  }
  __syncthreads();
  for (int p = t; p < nprobe; p += 256)
    probe[(size_t)q * nprobe + p] =
        s_fall ? centroid_probe[(size_t)q * nprobe + p] : (int32_t)(uint32_t)(pick[p] & 0xFFFFFFFFu);
}

}  // namespace

struct Router {
  int device = 0, num_sms = 148;
  uint32_t d = 0, h1 = 0, h2 = 0, G = 0, max_batch = 0;
  uint64_t step = 0;
  // parameters: FP32 masters, gradients, Adam moments, BF16 copies
  float* W[6] = {};
  float* dW[6] = {};
  float* m[6] = {};
  float* v[6] = {};
  size_t n[6] = {};
  uint16_t *W1b = nullptr, *W2b = nullptr, *W3b = nullptr, *W2bT = nullptr, *W3bT = nullptr;
  // activations for up to max_batch rows
  uint16_t *Xb = nullptr, *XbT = nullptr, *H1b = nullptr, *H1bT = nullptr, *H2b = nullptr, *H2bT = nullptr;
  float *A1 = nullptr, *A2 = nullptr, *L = nullptr, *dL = nullptr, *dH2 = nullptr, *dA2 = nullptr, *dH1 = nullptr,
        *dA1 = nullptr;
  uint16_t *dLb = nullptr, *dLbT = nullptr, *dA2b = nullptr, *dA2bT = nullptr, *dA1b = nullptr, *dA1bT = nullptr;
  float *mx = nullptr, *sm = nullptr;
  int* d_err = nullptr;
  // AdamW step count and its bias corrections (1 - b1^t, 1 - b2^t), kept on
  // the device so that one captured training step stays valid for every step
  unsigned long long* d_step = nullptr;
  float* d_bc = nullptr;
  // the training step as a CUDA graph, captured on a private stream and
  // re-captured (then updated in place) when its arguments change
  bool graphs = true;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec = nullptr;
  struct StepArgs {
    const float* X;
    const float* T;
    float* loss;
    uint32_t B;
    float lr, wd;
    int update;
    bool operator==(const StepArgs& o) const {
      return X == o.X && T == o.T && loss == o.loss && B == o.B && lr == o.lr && wd == o.wd && update == o.update;
    }
  } gargs{};
  std::vector<void*> allocs;
};

namespace {

int ralloc(Router& R, void** p, size_t bytes) {
  if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) return fail(HNTL_ENOMEM, "router allocation");
  R.allocs.push_back(*p);
  return HNTL_OK;
}

void rfree(Router& R) {
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(R.device);
  if (R.gexec) cudaGraphExecDestroy(R.gexec);
  if (R.cap) cudaStreamDestroy(R.cap);
  R.gexec = nullptr;
  R.cap = nullptr;
  for (void* p : R.allocs) cudaFree(p);
  R.allocs.clear();
  if (prev >= 0) cudaSetDevice(prev);
}

int gemm(const Router& R, const uint16_t* A, const uint16_t* B, int M, int N, int K, GemmEpi epi, cudaStream_t st) {
  // 64-wide tiles where 128-wide ones would not give every SM a CTA
  const bool narrow = (size_t)((N + kGTN - 1) / kGTN) * ((M + kGTM - 1) / kGTM) < (size_t)R.num_sms;
  const int bn = narrow ? 64 : 128;
  CUtensorMap ma, mb;
  if (!make_tma_map(&ma, A, true, (uint64_t)M, (uint64_t)K, kGTM) ||
      !make_tma_map(&mb, B, true, (uint64_t)N, (uint64_t)K, (uint32_t)bn))
    return fail(HNTL_ECUDA, "router: cannot encode TMA maps");
  dim3 grid((N + bn - 1) / bn, (M + kGTM - 1) / kGTM);
  if (narrow)
    k_gemm_tn<64><<<grid, 128, gemm_smem<64>(), st>>>(ma, mb, M, N, K, epi, R.d_err);
  else
    k_gemm_tn<128><<<grid, 128, gemm_smem<128>(), st>>>(ma, mb, M, N, K, epi, R.d_err);
  HNTL_CUDA_TRY(cudaGetLastError());
  return HNTL_OK;
}

void transpose(const uint16_t* src, int rows, int cols, uint16_t* dst, cudaStream_t st) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32);
  k_transpose_bf16<<<grid, dim3(32, 8), 0, st>>>(src, rows, cols, dst);
}

void colsum(const float* x, int rows, int cols, float* out, cudaStream_t st) {
  k_colsum<<<(cols + 31) / 32, dim3(32, kColGroups), 0, st>>>(x, rows, cols, out);
}

void to_bf16(const float* x, size_t n, uint16_t* y, cudaStream_t st) {
  k_f32_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, n, y);
}

void refresh_bf16(Router& R, cudaStream_t st) {
  to_bf16(R.W[0], R.n[0], R.W1b, st);
  to_bf16(R.W[2], R.n[2], R.W2b, st);
  to_bf16(R.W[4], R.n[4], R.W3b, st);
  transpose(R.W2b, R.h2, R.h1, R.W2bT, st);
  transpose(R.W3b, R.G, R.h2, R.W3bT, st);
}

// The MLP's forward pass into R.L. With train, the FP32 pre-activations A1, A2
// are kept for the GELU backward; inference writes only the BF16 activations.
int forward(Router& R, const float* X, uint32_t B, cudaStream_t st, bool train = true) {
  int rc;
  to_bf16(X, (size_t)B * R.d, R.Xb, st);
  if ((rc = gemm(R, R.Xb, R.W1b, (int)B, (int)R.h1, (int)R.d,
                 GemmEpi{train ? R.A1 : nullptr, R.H1b, R.W[1], 1, (int)R.h1}, st)))
    return rc;
  if ((rc = gemm(R, R.H1b, R.W2b, (int)B, (int)R.h2, (int)R.h1,
                 GemmEpi{train ? R.A2 : nullptr, R.H2b, R.W[3], 1, (int)R.h2}, st)))
    return rc;
  return gemm(R, R.H2b, R.W3b, (int)B, (int)R.G, (int)R.h2, GemmEpi{R.L, nullptr, R.W[5], 0, (int)R.G}, st);
}

int check_dims(uint32_t d, uint32_t h1, uint32_t h2, uint32_t G, uint32_t B) {
  if (!d || !h1 || !h2 || !G || !B) return fail(HNTL_EINVAL, "router sizes must be positive");
  if (d % 8 || h1 % 8 || h2 % 8 || G % 8 || B % 8)
    return fail(HNTL_EINVAL, "router sizes and batch must be multiples of 8 (16-byte BF16 rows)");
  return HNTL_OK;
}

}  // namespace

int router_route_probes(Router& R, const Index& I, const float* Q, uint32_t nq, uint32_t nprobe, float tau,
                        void* ws, size_t ws_bytes, int32_t* probe, uint32_t* nfallback, cudaStream_t st);

}  // namespace hntl

struct hntl_router {
  hntl::Router R;
};

using hntl::fail;

extern "C" int hntl_router_create(int device, uint32_t d, uint32_t h1, uint32_t h2, uint32_t G, uint32_t max_batch,
                                  const float* h_W1, const float* h_b1, const float* h_W2, const float* h_b2,
                                  const float* h_W3, const float* h_b3, hntl_router** out) {
  hntl::clear_error();
  if (!out) return fail(HNTL_EINVAL, "null argument");
  *out = nullptr;
  int rc = hntl::check_dims(d, h1, h2, G, max_batch);
  if (rc) return rc;
  const float* init[6] = {h_W1, h_b1, h_W2, h_b2, h_W3, h_b3};
  for (auto p : init)
    if (!p) return fail(HNTL_EINVAL, "initial parameters are required");
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return fail(HNTL_ECUDA, "cannot select the device");
  hntl_router* h = new (std::nothrow) hntl_router();
  if (!h) return fail(HNTL_ENOMEM, "host allocation");
  hntl::Router& R = h->R;
  R.device = device;
  R.d = d;
  R.h1 = h1;
  R.h2 = h2;
  R.G = G;
  R.max_batch = max_batch;
  const size_t n[6] = {(size_t)h1 * d, h1, (size_t)h2 * h1, h2, (size_t)G * h2, G};
  const size_t B = max_batch;
  do {
    for (int i = 0; i < 6; ++i) {
      R.n[i] = n[i];
      if ((rc = hntl::ralloc(R, (void**)&R.W[i], n[i] * 4)) || (rc = hntl::ralloc(R, (void**)&R.dW[i], n[i] * 4)) ||
          (rc = hntl::ralloc(R, (void**)&R.m[i], n[i] * 4)) || (rc = hntl::ralloc(R, (void**)&R.v[i], n[i] * 4)))
        break;
    }
    if (rc) break;
    void** b16[] = {(void**)&R.W1b, (void**)&R.W2b, (void**)&R.W3b, (void**)&R.W2bT, (void**)&R.W3bT};
    const size_t b16n[] = {n[0], n[2], n[4], n[2], n[4]};
    for (int i = 0; i < 5 && !rc; ++i) rc = hntl::ralloc(R, b16[i], b16n[i] * 2);
    if (rc) break;
    struct {
      void** p;
      size_t bytes;
    } acts[] = {{(void**)&R.Xb, B * d * 2},      {(void**)&R.XbT, B * d * 2},    {(void**)&R.H1b, B * h1 * 2},
                {(void**)&R.H1bT, B * h1 * 2},   {(void**)&R.H2b, B * h2 * 2},   {(void**)&R.H2bT, B * h2 * 2},
                {(void**)&R.A1, B * h1 * 4},     {(void**)&R.A2, B * h2 * 4},    {(void**)&R.L, B * G * 4},
                {(void**)&R.dL, B * G * 4},      {(void**)&R.dH2, B * h2 * 4},   {(void**)&R.dA2, B * h2 * 4},
                {(void**)&R.dH1, B * h1 * 4},    {(void**)&R.dA1, B * h1 * 4},   {(void**)&R.dLb, B * G * 2},
                {(void**)&R.dLbT, B * G * 2},    {(void**)&R.dA2b, B * h2 * 2},  {(void**)&R.dA2bT, B * h2 * 2},
                {(void**)&R.dA1b, B * h1 * 2},   {(void**)&R.dA1bT, B * h1 * 2}, {(void**)&R.mx, B * 4},
                {(void**)&R.sm, B * 4},          {(void**)&R.d_err, 4},          {(void**)&R.d_step, 8},
                {(void**)&R.d_bc, 8}};
    for (auto& a : acts)
      if ((rc = hntl::ralloc(R, a.p, a.bytes))) break;
    if (rc) break;
    for (int i = 0; i < 6 && !rc; ++i) {
      if (cudaMemcpy(R.W[i], init[i], n[i] * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemset(R.m[i], 0, n[i] * 4) != cudaSuccess || cudaMemset(R.v[i], 0, n[i] * 4) != cudaSuccess ||
          cudaMemset(R.dW[i], 0, n[i] * 4) != cudaSuccess)
        rc = fail(HNTL_ECUDA, "router: parameter upload");
    }
    if (rc) break;
    cudaMemset(R.d_err, 0, 4);
    cudaMemset(R.d_step, 0, 8);
    hntl::refresh_bf16(R, nullptr);
    // set up here, never while a step is being captured
    CUtensorMap probe_map;
    if (cudaFuncSetAttribute(hntl::k_gemm_tn<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             hntl::gemm_smem<128>()) != cudaSuccess ||
        cudaFuncSetAttribute(hntl::k_gemm_tn<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             hntl::gemm_smem<64>()) != cudaSuccess ||
        cudaDeviceGetAttribute(&R.num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        !hntl::make_tma_map(&probe_map, R.W1b, true, h1, d, hntl::kGTN) ||
        cudaStreamCreateWithFlags(&R.cap, cudaStreamNonBlocking) != cudaSuccess) {
      rc = fail(HNTL_ECUDA, "router: GEMM set-up");
      break;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) rc = fail(HNTL_ECUDA, "router: initialisation");
  } while (0);
  if (prev >= 0) cudaSetDevice(prev);
  if (rc) {
    hntl::rfree(R);
    delete h;
    return rc;
  }
  *out = h;
  return HNTL_OK;
}

extern "C" void hntl_router_free(hntl_router* h) {
  if (!h) return;
  hntl::rfree(h->R);
  delete h;
}

static int copy_out(const hntl::Router& R, float* const* dst, float* const* src) {
  for (int i = 0; i < 6; ++i)
    if (dst[i] && cudaMemcpy(dst[i], src[i], R.n[i] * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(HNTL_ECUDA, "router: copy to host");
  return HNTL_OK;
}

extern "C" int hntl_router_params(const hntl_router* h, float* W1, float* b1, float* W2, float* b2, float* W3,
                                  float* b3) {
  hntl::clear_error();
  if (!h) return fail(HNTL_EINVAL, "null router");
  float* dst[6] = {W1, b1, W2, b2, W3, b3};
  return copy_out(h->R, dst, h->R.W);
}

extern "C" int hntl_router_grads(const hntl_router* h, float* dW1, float* db1, float* dW2, float* db2, float* dW3,
                                 float* db3) {
  hntl::clear_error();
  if (!h) return fail(HNTL_EINVAL, "null router");
  float* dst[6] = {dW1, db1, dW2, db2, dW3, db3};
  return copy_out(h->R, dst, h->R.dW);
}

namespace hntl {
namespace {

// Every launch of one training step, in order, on `st`.
int enqueue_step(Router& R, const float* d_X, const float* d_T, uint32_t B, float lr, float wd, int update,
                 float* d_loss, cudaStream_t st) {
  int rc;
  if ((rc = forward(R, d_X, B, st))) return rc;
  k_softmax_ce<<<B, 256, 0, st>>>(R.L, d_T, (int)R.G, (int)B, R.dL, R.dLb, d_loss);
  // output layer
  transpose(R.dLb, (int)B, (int)R.G, R.dLbT, st);
  transpose(R.H2b, (int)B, (int)R.h2, R.H2bT, st);
  if ((rc = gemm(R, R.dLbT, R.H2bT, (int)R.G, (int)R.h2, (int)B, GemmEpi{R.dW[4], nullptr, nullptr, 0, (int)R.h2}, st)))
    return rc;
  colsum(R.dL, (int)B, (int)R.G, R.dW[5], st);
  if ((rc = gemm(R, R.dLb, R.W3bT, (int)B, (int)R.h2, (int)R.G, GemmEpi{R.dH2, nullptr, nullptr, 0, (int)R.h2}, st)))
    return rc;
  // second hidden layer
  const size_t n2 = (size_t)B * R.h2, n1 = (size_t)B * R.h1;
  k_gelu_bwd<<<(unsigned)((n2 + 255) / 256), 256, 0, st>>>(R.dH2, R.A2, n2, R.dA2, R.dA2b);
  transpose(R.dA2b, (int)B, (int)R.h2, R.dA2bT, st);
  transpose(R.H1b, (int)B, (int)R.h1, R.H1bT, st);
  if ((rc = gemm(R, R.dA2bT, R.H1bT, (int)R.h2, (int)R.h1, (int)B, GemmEpi{R.dW[2], nullptr, nullptr, 0, (int)R.h1}, st)))
    return rc;
  colsum(R.dA2, (int)B, (int)R.h2, R.dW[3], st);
  if ((rc = gemm(R, R.dA2b, R.W2bT, (int)B, (int)R.h1, (int)R.h2, GemmEpi{R.dH1, nullptr, nullptr, 0, (int)R.h1}, st)))
    return rc;
  // first hidden layer
  k_gelu_bwd<<<(unsigned)((n1 + 255) / 256), 256, 0, st>>>(R.dH1, R.A1, n1, R.dA1, R.dA1b);
  transpose(R.dA1b, (int)B, (int)R.h1, R.dA1bT, st);
  transpose(R.Xb, (int)B, (int)R.d, R.XbT, st);
  if ((rc = gemm(R, R.dA1bT, R.XbT, (int)R.h1, (int)R.d, (int)B, GemmEpi{R.dW[0], nullptr, nullptr, 0, (int)R.d}, st)))
    return rc;
  colsum(R.dA1, (int)B, (int)R.h1, R.dW[1], st);
  if (update) {
    constexpr float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    k_adam_tick<<<1, 1, 0, st>>>(R.d_step, R.d_bc, b1, b2);
    AdamSet S{};
    unsigned nb = 0;
    for (int i = 0; i < 6; ++i) {
      S.p[i] = R.W[i];
      S.g[i] = R.dW[i];
      S.m[i] = R.m[i];
      S.v[i] = R.v[i];
      S.pb[i] = i == 0 ? R.W1b : i == 2 ? R.W2b : i == 4 ? R.W3b : nullptr;
      S.n[i] = R.n[i];
      S.wd[i] = (i % 2 == 0) ? wd : 0.f;  // decay on the weight matrices only
      S.blk[i] = nb;
      nb += (unsigned)((R.n[i] + 255) / 256);
    }
    S.blk[6] = nb;
    k_adamw<<<nb, 256, 0, st>>>(S, lr, b1, b2, eps, R.d_bc);
    transpose(R.W2b, (int)R.h2, (int)R.h1, R.W2bT, st);
    transpose(R.W3b, (int)R.G, (int)R.h2, R.W3bT, st);
  }
  HNTL_CUDA_TRY(cudaGetLastError());
  return HNTL_OK;
}

// Captures the step for `a` on the private stream and makes R.gexec run it:
// updated in place when the graph's shape allows, else instantiated anew.
int capture_step(Router& R, const Router::StepArgs& a) {
  HNTL_CUDA_TRY(cudaStreamBeginCapture(R.cap, cudaStreamCaptureModeThreadLocal));
  const int rc = enqueue_step(R, a.X, a.T, a.B, a.lr, a.wd, a.update, a.loss, R.cap);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(R.cap, &g);
  if (rc || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (rc) return rc;
    return fail(HNTL_ECUDA, std::string("router: step capture: ") + cudaGetErrorString(e));
  }
  if (R.gexec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(R.gexec, g, &info) != cudaSuccess) {
      (void)cudaGetLastError();  // not updatable (e.g. other grid sizes): instantiate below
      cudaGraphExecDestroy(R.gexec);
      R.gexec = nullptr;
    }
  }
  cudaError_t ie = cudaSuccess;
  if (!R.gexec) ie = cudaGraphInstantiate(&R.gexec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    R.gexec = nullptr;
    return fail(HNTL_ECUDA, std::string("router: step graph: ") + cudaGetErrorString(ie));
  }
  R.gargs = a;
  return HNTL_OK;
}

}  // namespace
}  // namespace hntl

extern "C" int hntl_router_step(hntl_router* h, const float* d_X, const float* d_T, uint32_t B, float lr, float wd,
                                int update, float* d_loss, void* stream) {
  hntl::clear_error();
  if (!h || !d_X || !d_T) return fail(HNTL_EINVAL, "null argument");
  hntl::Router& R = h->R;
  int rc = hntl::check_dims(R.d, R.h1, R.h2, R.G, B);
  if (rc) return rc;
  if (B > R.max_batch) return fail(HNTL_EINVAL, "batch larger than the router's max_batch");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!R.graphs) return hntl::enqueue_step(R, d_X, d_T, B, lr, wd, update, d_loss, st);
  const hntl::Router::StepArgs a{d_X, d_T, d_loss, B, lr, wd, update};
  if (!R.gexec || !(a == R.gargs))
    if ((rc = hntl::capture_step(R, a))) return rc;
  HNTL_CUDA_TRY(cudaGraphLaunch(R.gexec, st));
  return HNTL_OK;
}

extern "C" int hntl_router_set_graphs(hntl_router* h, int enable) {
  hntl::clear_error();
  if (!h) return fail(HNTL_EINVAL, "null router");
  h->R.graphs = enable != 0;
  return HNTL_OK;
}

extern "C" int hntl_router_status(const hntl_router* h) {
  hntl::clear_error();
  if (!h) return fail(HNTL_EINVAL, "null router");
  int e = 0;
  HNTL_CUDA_TRY(cudaMemcpy(&e, h->R.d_err, sizeof(int), cudaMemcpyDeviceToHost));
  return e ? fail(HNTL_ETIMEOUT, "router: a tensor-core pipeline wait timed out") : HNTL_OK;
}

extern "C" int hntl_router_logits(hntl_router* h, const float* d_X, uint32_t B, float* d_logits, void* stream) {
  hntl::clear_error();
  if (!h || !d_X || !d_logits) return fail(HNTL_EINVAL, "null argument");
  hntl::Router& R = h->R;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (uint32_t s = 0; s < B; s += R.max_batch) {
    const uint32_t b = std::min(R.max_batch, B - s);
    int rc = hntl::check_dims(R.d, R.h1, R.h2, R.G, (b + 7) / 8 * 8);
    if (rc) return rc;
    if ((rc = hntl::forward(R, d_X + (size_t)s * R.d, b, st, false))) return rc;
    HNTL_CUDA_TRY(cudaMemcpyAsync(d_logits + (size_t)s * R.G, R.L, sizeof(float) * b * R.G, cudaMemcpyDeviceToDevice, st));
  }
  return HNTL_OK;
}

namespace hntl {

// Router probes (the nprobe largest logits) for every query; where their
// softmax mass is below tau, the query's centroid probes instead. Workspace:
// as hntl_search_workspace_bytes(idx, nq, 1, 1, nprobe) for the centroid
// routing, then nq * nprobe int32 + nq * nprobe floats + nq * G floats.
int router_route_probes(Router& R, const Index& I, const float* Q, uint32_t nq, uint32_t nprobe, float tau,
                        void* ws, size_t ws_bytes, int32_t* probe, uint32_t* nfallback, cudaStream_t st) {
  if (R.G != I.G || R.d != I.d) return fail(HNTL_EINVAL, "router and index disagree on d or G");
  if (nprobe < 1 || nprobe > I.G) return fail(HNTL_EINVAL, "nprobe must be in [1, G]");
  const size_t route_ws = workspace_bytes(I, nq, 1, 1, nprobe);
  if (!route_ws) return HNTL_EINVAL;
  Carver c(static_cast<char*>(ws) + route_ws);
  int32_t* cprobe = c.take<int32_t>((size_t)nq * nprobe);
  float* cdist = c.take<float>((size_t)nq * nprobe);
  float* negl = c.take<float>((size_t)nq * I.G);
  float* negtop = c.take<float>((size_t)nq * nprobe);
  if (ws_bytes < route_ws + align_up(c.off, 256)) return fail(HNTL_EINVAL, "router routing workspace too small");
  // the fused selection for up to kTopMax probes; with tau <= 0 no query falls
  // back there, so the centroid probes are not computed at all
  const bool fused = nprobe <= (uint32_t)kTopMax && I.G <= 256u * 32u;
  const bool centroid = !fused || tau > 0.f;
  int rc = HNTL_OK;
  if (centroid && (rc = route_only(I, Q, nq, nprobe, ws, route_ws, cprobe, cdist, st))) return rc;
  if (nfallback) HNTL_CUDA_TRY(cudaMemsetAsync(nfallback, 0, 4, st));
  static thread_local int attr_dev = -1;  // device whose select attribute this thread has set
  if (attr_dev != I.device) {
    HNTL_CUDA_TRY(cudaFuncSetAttribute(k_route_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSelWarps * (int)kMaxG * (int)sizeof(float)));
    attr_dev = I.device;
  }
  for (uint32_t s = 0; s < nq; s += R.max_batch) {
    const uint32_t b = std::min(R.max_batch, nq - s);
    if ((rc = forward(R, Q + (size_t)s * R.d, b, st, false))) return rc;
    if (fused) {
      const int32_t* cp = centroid ? cprobe + (size_t)s * nprobe : nullptr;
      if (R.G <= 256 * 16)
        k_router_topk<16><<<b, 256, 0, st>>>(R.L, (int)R.G, (int)nprobe, tau, cp, probe + (size_t)s * nprobe,
                                             nfallback);
      else
        k_router_topk<32><<<b, 256, 0, st>>>(R.L, (int)R.G, (int)nprobe, tau, cp, probe + (size_t)s * nprobe,
                                             nfallback);
      continue;
    }
    k_logit_stats<<<b, 256, 0, st>>>(R.L, (int)R.G, negl + (size_t)s * R.G, R.mx, R.sm);
    k_route_select<<<(b + kSelWarps - 1) / kSelWarps, kSelWarps * 32, (size_t)kSelWarps * R.G * sizeof(float), st>>>(
        negl + (size_t)s * R.G, (int)b, (int)R.G, (int)nprobe, probe + (size_t)s * nprobe, negtop + (size_t)s * nprobe);
    k_router_merge<<<(b + 127) / 128, 128, 0, st>>>((int)b, (int)nprobe, negtop + (size_t)s * nprobe, R.mx, R.sm, tau,
                                                    cprobe + (size_t)s * nprobe, probe + (size_t)s * nprobe, nfallback);
  }
  HNTL_CUDA_TRY(cudaGetLastError());
  return HNTL_OK;
}

}  // namespace hntl

extern "C" size_t hntl_router_route_workspace_bytes(const hntl_router* h, const hntl_index* idx, uint32_t nq,
                                                    uint32_t nprobe) {
  hntl::clear_error();
  if (!h || !idx) {
    fail(HNTL_EINVAL, "null argument");
    return 0;
  }
  const size_t route_ws = hntl::workspace_bytes(idx->I, nq, 1, 1, nprobe);
  if (!route_ws) return 0;
  hntl::Carver c(nullptr);
  c.take<int32_t>((size_t)nq * nprobe);
  c.take<float>((size_t)nq * nprobe);
  c.take<float>((size_t)nq * idx->I.G);
  c.take<float>((size_t)nq * nprobe);
  return route_ws + hntl::align_up(c.off, 256);
}

extern "C" int hntl_router_route(hntl_router* h, const hntl_index* idx, const float* d_Q, uint32_t nq,
                                 uint32_t nprobe, float tau, void* d_ws, size_t ws_bytes, int32_t* d_probe,
                                 uint32_t* d_nfallback, void* stream) {
  hntl::clear_error();
  if (!h || !idx || !d_Q || !d_ws || !d_probe) return fail(HNTL_EINVAL, "null argument");
  if (nq == 0) return HNTL_OK;
  return hntl::router_route_probes(h->R, idx->I, d_Q, nq, nprobe, tau, d_ws, ws_bytes, d_probe, d_nfallback,
                                   static_cast<cudaStream_t>(stream));
}
