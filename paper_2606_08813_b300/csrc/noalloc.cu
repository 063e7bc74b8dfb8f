// Allocation-free centroid routing: hntl_route_noalloc.
//
// Some callers cannot allocate device memory when they query: a host
// application that reserves the whole GPU at start-up and gives its plug-ins
// no allocator, or a latency-critical loop where a cudaMalloc would
// synchronise the device. For them this entry point routes a batch without
// any workspace from the caller and without allocating: its scratch (the
// nq x G distance matrix) is a file-scope device array of fixed size that
// every GPU which loads the library holds until the process exits.
//
// The array's name in host code is a host-side stand-in, not a device
// address, so the device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached. That happens on
// the first call on each device, so make the first call on a device before
// any stream capture begins. All calls share the one array and each call
// overwrites the part it uses before reading it (nothing needs to start at
// zero); two calls whose kernels overlap on the GPU (different streams,
// different host threads) race on it.
#include <mutex>
#include <string>

#include "hntl_internal.cuh"
#include "route_kernels.cuh"

namespace hntl {
namespace {

// Largest nq * G a call may route: 2^21 distances (8 MiB of device memory).
constexpr size_t kNoAllocRouteFloats = size_t(1) << 21;
static __device__ __align__(256) float g_route_scratch[kNoAllocRouteFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current).
int scratch_on(int device, float** out) {
  if (device < 0 || device >= kMaxDevices) return fail(HNTL_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_route_scratch);
    if (e != cudaSuccess)
      return fail(HNTL_ECUDA, std::string("cudaGetSymbolAddress(route scratch): ") + cudaGetErrorString(e));
    e = cudaFuncSetAttribute(k_route_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSelWarps * (int)kMaxG * (int)sizeof(float));
    if (e != cudaSuccess)
      return fail(HNTL_ECUDA, std::string("cudaFuncSetAttribute(route select): ") + cudaGetErrorString(e));
    g_scratch_ptr[device] = static_cast<float*>(p);
  }
  *out = g_scratch_ptr[device];
  return HNTL_OK;
}

}  // namespace
}  // namespace hntl

extern "C" int hntl_route_noalloc(const hntl_index* idx, const float* d_queries, uint32_t nq, uint32_t nprobe,
                                  int32_t* d_probe, float* d_probe_dist, void* stream) {
  hntl::clear_error();
  if (!idx) return hntl::fail(HNTL_EINVAL, "null index");
  const hntl::Index& I = idx->I;
  if (nprobe < 1 || nprobe > I.G) return hntl::fail(HNTL_EINVAL, "nprobe must be in [1, G]");
  if (I.precision != HNTL_PREC_FP32)
    return hntl::fail(HNTL_EINVAL, "allocation-free routing serves FP32 indices only");
  if ((size_t)nq * I.G > hntl::kNoAllocRouteFloats)
    return hntl::fail(HNTL_EINVAL, "nq * G = " + std::to_string((size_t)nq * I.G) +
                                       " exceeds the allocation-free routing limit of " +
                                       std::to_string(hntl::kNoAllocRouteFloats) + " distances");
  if (nq == 0) return HNTL_OK;
  if (!d_queries || !d_probe || !d_probe_dist) return hntl::fail(HNTL_EINVAL, "null buffer");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != I.device && cudaSetDevice(I.device) != cudaSuccess)
    return hntl::fail(HNTL_ECUDA, "cannot make the index's device current");
  float* scratch = nullptr;
  int rc = hntl::scratch_on(I.device, &scratch);
  if (rc == HNTL_OK) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    dim3 grid((I.G + hntl::kRT - 1) / hntl::kRT, (nq + hntl::kRT - 1) / hntl::kRT);
    hntl::k_route_dist<<<grid, 256, 0, st>>>(d_queries, I.M, (int)nq, (int)I.G, (int)I.d, scratch);
    size_t smem = (size_t)hntl::kSelWarps * I.G * sizeof(float);
    hntl::k_route_select<<<(nq + hntl::kSelWarps - 1) / hntl::kSelWarps, hntl::kSelWarps * 32, smem, st>>>(
        scratch, (int)nq, (int)I.G, (int)nprobe, d_probe, d_probe_dist);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = hntl::fail(HNTL_ECUDA, std::string("route launch: ") + cudaGetErrorString(e));
  }
  if (prev >= 0 && prev != I.device) cudaSetDevice(prev);
  return rc;
}
