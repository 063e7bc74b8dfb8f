// Internal declarations of the HNTL CUDA library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hntl.h"

namespace hntl {

// Rows per Block-SoA block: one thread per row in the scan, 128-row tiles.
constexpr int kBlockRows = 128;
constexpr int kMaxR = 64;
constexpr int kMaxC = 1024;
constexpr uint32_t kMaxG = 8192;
constexpr uint32_t kInvalidId = 0xFFFFFFFFu;

// Block-SoA with 16-byte lanes. Grains are stored one after another, each
// padded to whole 128-row blocks. Inside a block the coordinates are
// dimension-major in lanes of V = 16 bytes (4 FP32 or 16 FP8 coordinates):
// lane c of row t of block b holds coordinates cV .. cV+V-1 at
//   ((b * rp/V + c) * 128 + t) * V,
// with rp = r rounded up to V (zero padding). A thread (one row) reads its row
// with rp/V 16-byte loads and a warp's load covers 512 contiguous bytes.
// Padding rows carry id 0xFFFFFFFF and are masked by the grain's row count.
// Coordinate storage kinds (equal to the HNTL_PREC_* value of the index).
constexpr int kCoordF32 = 0, kCoordFP8 = 1, kCoordI16 = 2;
// Coordinates per 16-byte lane of the Block-SoA layout.
__host__ __device__ inline int coord_lane(int kind) { return kind == kCoordFP8 ? 16 : (kind == kCoordI16 ? 8 : 4); }
__host__ __device__ inline int padded_r(int r, int kind) {
  const int V = coord_lane(kind);
  return (r + V - 1) / V * V;
}
__host__ __device__ inline size_t zoff(size_t b, int j, int t, int rp, int V) {
  return ((b * (size_t)(rp / V) + (size_t)(j / V)) * 128 + (size_t)t) * V + (size_t)(j % V);
}
struct Index {
  int device = 0;
  uint64_t n = 0;
  uint32_t d = 0, G = 0, r = 0, precision = HNTL_PREC_FP32;
  uint32_t rp = 0;               // r padded to the coordinate lane (see zoff)
  bool has_attr = false;
  bool i16_resid_prune = false;  // 16-bit form: also leave a grain out when the query residual saturates
  uint64_t n_blocks = 0;
  uint64_t max_grain_rows = 0;
  uint64_t device_bytes = 0;

  float* M = nullptr;            // [G][d] centres
  float* U = nullptr;            // [G][r][d] bases, orthonormal rows
  uint32_t* blk_off = nullptr;   // [G+1] first block of each grain
  uint32_t* grain_rows = nullptr;  // [G] rows of each grain
  uint32_t* blk_grain = nullptr;   // [n_blocks] grain of each block
  float* Zb = nullptr;           // [n_blocks][rp/4][128][4] FP32 coordinates
  uint8_t* Z8b = nullptr;        // [n_blocks][rp/16][128][16] FP8-E4M3 codes (precision form)
  int16_t* Z16b = nullptr;       // [n_blocks][rp/8][128][8] int16 codes (16-bit form)
  float* scale = nullptr;        // [G] FP8 scale, or the 16-bit form's coordinate step, per grain
  float* dres = nullptr;         // [G] the 16-bit form's residual step per grain
  float* rho = nullptr;          // [n_blocks][128] residual norms
  float* blk_rho_min = nullptr;  // [n_blocks] smallest residual norm of a block's real rows (+inf if none)
  float2* blk_z0 = nullptr;      // [n_blocks] [min, max] of the decoded first coordinate of a block's real rows
  float* crow = nullptr;         // [n_blocks][128] ||z_i||^2 + rho_i of the decoded row (precision form)
  float* grain_rho_min = nullptr;  // [G] smallest residual norm of a grain's rows (precision form)
  uint32_t* ids = nullptr;       // [n_blocks][128] original ids
  int64_t* attr_b = nullptr;     // [n_blocks][128] attributes in block order
  uint32_t* gid = nullptr;       // [n] a grain shard's original id of each local row (nullptr: not a shard)
  float* X = nullptr;            // [n][d] FP32 raw rows, id order
  uint16_t* Xh = nullptr;        // [n][d] BF16 raw rows, id order
  uint16_t* Xl = nullptr;        // [n][d] second BF16 parts bf16(x - bf16(x)) (refined rerank), or nullptr

  // derived at load/build (finalize_index)
  float* mnorm = nullptr;        // [G] ||mu_g||^2 (of the BF16 centres in the precision form)
  uint16_t* Mh = nullptr;        // [G][d] BF16 centres (precision form)
  uint16_t* Mhn = nullptr;       // [G][d] the same negated (the projection's -mu_b operand)
  int num_sms = 148;             // streaming multiprocessors of the index's device
  uint16_t* Uh = nullptr;        // [G][r][d] BF16 bases (precision form)
  float* gram = nullptr;         // [G][r][r] U_g U_g^T (of the BF16 bases in the precision form)
  uint32_t* pos_of_id = nullptr; // [n] stored position (block * 128 + row) of each id (Mode A)
  float* hrow = nullptr;         // [n_blocks][128] z_i^T G_g z_i of the decoded row (Mode A)
  int* d_err = nullptr;          // device error word (bounded waits that gave up)
  bool tc_route = false;         // tensor-core routing available (TMA map built)
  CUtensorMap mapM;              // TMA map of the centres (FP32 or BF16), 256-row boxes
  CUtensorMap mapU;              // precision form: bases (r-row box)
  bool tc_proj = false;
  uint16_t* U3 = nullptr;        // [3][G][r][d] BF16 parts of the FP32 bases (FP32 and 16-bit forms)
  CUtensorMap mapU3;             // their TMA map (3 G r rows, r-row box)
  bool tc_proj32 = false;        // FP32-accurate tensor-core projection available (r <= 32)

  // host copies used for workspace sizing
  std::vector<uint32_t> h_blk_off;
  std::vector<uint64_t> h_top_padded_prefix;  // prefix sums of padded grain sizes, largest first
  std::vector<void*> allocations;
};

// Frees an index's device memory (safe to call twice).
void release(Index& I);

// Derived device state after the arrays are in place (both loader and builder call it).
int finalize_index(Index& I);

// Grain-ordered row positions, each grain's rows sorted by (first coordinate,
// id): the order in which they are laid out into blocks (host code shared by
// loader and builder). Z: N x r grain-ordered; ids: their ids.
std::vector<uint64_t> rows_by_first_coord(const float* Z, uint32_t r, const uint32_t* ids,
                                          const std::vector<uint64_t>& goff);

// The 16-bit form (Eq. 5) of grain-ordered rows (Z: N x r, rho: N; goff: G + 1
// grain offsets), in IEEE single precision: per grain the steps
// delta = fl32(max |z| / 16383) and dres = fl32(R / 32767) with
// R = max(max rho, fl32(max|z|^2) 2^-20) (1 for a grain of zeros), codes
// rint(fl32(z / delta)), and rho on its grid,
// fl32(rint(fl32(rho / dres)) * dres). Host code shared by loader and builder.
void int16_quantize(const float* Z, const float* rho, const std::vector<uint64_t>& goff, uint32_t r,
                    std::vector<float>& delta, std::vector<float>& dres, std::vector<int16_t>& codes,
                    std::vector<float>& rho_q);

// Search internals shared with the router.
size_t workspace_bytes(const Index& I, uint32_t nq, uint32_t k, uint32_t C, uint32_t nprobe);
int route_only(const Index& I, const float* Qd, uint32_t nq, uint32_t nprobe, void* ws, size_t ws_bytes,
               int32_t* probe, float* probe_d, cudaStream_t st);

// TMA map of a row-major matrix [rows][d] (FP32 or BF16) with 128-byte K boxes.
bool make_tma_map(CUtensorMap* map, const void* base, bool bf16, uint64_t rows, uint64_t d, uint32_t box_rows);

// Thread-local error message plumbing.
int fail(int code, const std::string& msg);
void clear_error();

#define HNTL_CUDA_TRY(expr)                                                                  \
  do {                                                                                       \
    cudaError_t _e = (expr);                                                                 \
    if (_e != cudaSuccess)                                                                   \
      return ::hntl::fail(HNTL_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));   \
  } while (0)

// After a kernel launch: a launch error names the kernel.
#define HNTL_LAUNCH_CHECK(name)                                                              \
  do {                                                                                       \
    cudaError_t _e = cudaGetLastError();                                                     \
    if (_e != cudaSuccess)                                                                   \
      return ::hntl::fail(HNTL_ECUDA, std::string("launch of ") + (name) + ": " + cudaGetErrorString(_e)); \
  } while (0)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Workspace carving: every sub-buffer starts on a 256-byte boundary.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    off = align_up(off, 256);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

}  // namespace hntl

struct hntl_index {
  hntl::Index I;
};
