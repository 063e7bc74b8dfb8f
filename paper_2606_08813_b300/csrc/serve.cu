// Continuous-batching serving loop over one index.
//
// Requests are admitted into slots of a device-resident table (query row, k,
// C and attribute range stay on the device while the request lives). A host
// worker thread forms batches from the admitted requests as they arrive and
// launches them on one of kLanes lanes; each lane owns a stream, a workspace
// and CUDA graphs captured once at creation for the batch sizes B, B/2, B/4,
// ... down to 32 rows: gather the batch's slots from the table, run
// the whole Mode B search with each query's own k and C (k_max and C_max set
// the strides only), and copy the results to pinned host memory. A batch
// takes the smallest graph that holds it, padded with copies of its first
// request, so a lightly loaded server does not pay for full batches (at most
// twice the rows it holds). While lanes' batches run on the GPU the worker
// fills and launches the next free one, so requests that arrive meanwhile
// overlap with them.
// A request's result does not depend on the batch it rides in: every stage is
// per query (selections are total orders on (distance, id)).
//
// Memory admission: the budget first pays for the lanes (workspace and batch
// buffers); what remains sets how many requests can be held at once. A
// submission beyond the free slots is refused (its count of admitted
// requests is short), and the caller retries after polling.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstring>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hntl_internal.cuh"

namespace hntl {

int search(const Index& I, const float* Qd, uint32_t nq, uint32_t k, uint32_t C, uint32_t nprobe,
           const int64_t* filter, void* ws, size_t ws_bytes, int64_t* out_ids, float* out_d, uint32_t* cand_ids,
           float* cand_d, int32_t* probe_out, cudaStream_t st, const int32_t* probe_in, const uint32_t* qk,
           const uint32_t* qC, bool mode_a);

namespace {

__global__ void k_gather_batch(const uint32_t* __restrict__ slots, int B, int d, const float* __restrict__ slot_q,
                               const uint32_t* __restrict__ slot_k, const uint32_t* __restrict__ slot_C,
                               const int64_t* __restrict__ slot_range, float* __restrict__ Q, uint32_t* __restrict__ k,
                               uint32_t* __restrict__ C, int64_t* __restrict__ F) {
  const int i = blockIdx.x;
  if (i >= B) return;
  const uint32_t s = slots[i];
  if ((d & 3) == 0) {  // rows of whole 16-byte pieces: fewer, wider reads over the host link
    const float4* src = reinterpret_cast<const float4*>(slot_q + (size_t)s * d);
    float4* dst = reinterpret_cast<float4*>(Q + (size_t)i * d);
    for (int t = threadIdx.x; t < d / 4; t += blockDim.x) dst[t] = src[t];
  } else {
    for (int t = threadIdx.x; t < d; t += blockDim.x) Q[(size_t)i * d + t] = slot_q[(size_t)s * d + t];
  }
  if (threadIdx.x == 0) {
    k[i] = slot_k[s];
    C[i] = slot_C[s];
    if (F) {
      F[2 * i] = slot_range[2 * (size_t)s];
      F[2 * i + 1] = slot_range[2 * (size_t)s + 1];
    }
  }
}

using Clock = std::chrono::steady_clock;

// Latency histogram with log-linear buckets: nanosecond values below 64 are
// exact, above that each power of two splits into 64 buckets, so a quantile
// read from it is within 1/64 of the sample it stands for. Recording is O(1)
// and never allocates (it runs under the queue's lock).
struct LatencyHist {
  static constexpr int kSub = 64, kOctaves = 42;  // up to 2^47 ns
  static constexpr int kBuckets = kSub + kOctaves * kSub;
  uint64_t count[kBuckets] = {};
  uint64_t n = 0;
  int64_t max_ns = 0;
  static int bucket(int64_t v) {
    if (v < kSub) return (int)std::max<int64_t>(v, 0);
    const int e = 63 - __builtin_clzll((uint64_t)v);  // >= 6
    const int b = kSub + (e - 6) * kSub + (int)((v >> (e - 6)) & (kSub - 1));
    return std::min(b, kBuckets - 1);
  }
  static double middle(int b) {  // centre of bucket b, in ns
    if (b < kSub) return (double)b;
    const int e = (b - kSub) / kSub + 6, sub = (b - kSub) % kSub;
    const double lo = std::ldexp((double)(kSub + sub), e - 6);
    return lo + std::ldexp(0.5, e - 6);
  }
  void add(int64_t v) {
    ++count[bucket(v)];
    ++n;
    max_ns = std::max(max_ns, v);
  }
  void clear() {
    std::fill(count, count + kBuckets, 0);
    n = 0;
    max_ns = 0;
  }
  // the sample of rank floor(q (n - 1)) in ascending order, as microseconds
  double quantile_us(double q) const {
    if (!n) return 0.0;
    const uint64_t rank = (uint64_t)(q * (double)(n - 1));
    uint64_t seen = 0;
    for (int b = 0; b < kBuckets; ++b) {
      seen += count[b];
      if (seen > rank) return std::min(middle(b), (double)max_ns) / 1e3;
    }
    return (double)max_ns / 1e3;
  }
};

struct Req {
  uint32_t slot = 0, k = 0;
  int state = 0;  // 1 queued, 2 running, 3 done
  int64_t arrival_ns = 0;
  int64_t enter_ns = 0;   // its submission call began
  int64_t admit_ns = 0;   // entered the queue (its row copied into its slot)
  int64_t launch_ns = 0;  // its batch was launched
  std::vector<int64_t> ids;
  std::vector<float> dist;
};

struct Lane {
  cudaStream_t st = nullptr;
  std::vector<std::pair<uint32_t, cudaGraphExec_t>> graphs;  // (rows, graph), ascending rows
  cudaEvent_t done = nullptr;
  uint32_t* d_slots = nullptr;
  uint32_t* h_slots = nullptr;  // pinned
  float* d_Q = nullptr;
  uint32_t *d_k = nullptr, *d_C = nullptr;
  int64_t* d_F = nullptr;
  int64_t* d_ids = nullptr;
  float* d_dist = nullptr;
  int64_t* h_ids = nullptr;  // pinned
  float* h_dist = nullptr;   // pinned
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // the running batch's requests: a running request's entry is never
  // erased (only finished ones are), so these stay valid until it retires
  std::vector<Req*> reqs;
  bool busy = false;
};

constexpr int kLanes = 3;

}  // namespace

struct Server {
  const Index* I = nullptr;
  uint32_t B = 0, nprobe = 0, kmax = 0, Cmax = 0, nslots = 0;
  // the slot table lives in mapped pinned host memory: a submission writes its
  // rows with plain host stores (no CUDA call, so it never waits behind the
  // lanes' kernels) and each batch's gather kernel reads them over the host link
  float* h_slot_q = nullptr;
  uint32_t *h_slot_k = nullptr, *h_slot_C = nullptr;
  int64_t* h_slot_range = nullptr;
  float* d_slot_q = nullptr;  // device views of the same memory
  uint32_t *d_slot_k = nullptr, *d_slot_C = nullptr;
  int64_t* d_slot_range = nullptr;
  Lane lanes[kLanes];
  std::vector<void*> dev, host;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::vector<uint32_t> free_slots;
  std::unordered_map<uint64_t, Req> reqs;
  uint64_t next_ticket = 1;
  std::thread worker;
  std::atomic<bool> stop{false};
  LatencyHist lat, lag, upload, queue_wait, service;
  uint64_t batches = 0, batched = 0;
  std::atomic<int> worker_error{HNTL_OK};  // set by the worker, read by any thread
};

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

// Copy a finished batch's results into its requests (without the lock: only
// the worker touches a running request), then retire it under the lock.
void fill_results(Server& S, Lane& L) {
  for (size_t i = 0; i < L.reqs.size(); ++i) {
    Req& r = *L.reqs[i];
    r.ids.assign(L.h_ids + i * S.kmax, L.h_ids + i * S.kmax + r.k);
    r.dist.assign(L.h_dist + i * S.kmax, L.h_dist + i * S.kmax + r.k);
  }
}

void retire(Server& S, Lane& L) {
  // called with S.mu held, after fill_results
  const int64_t t = now_ns();
  for (Req* rp : L.reqs) {
    Req& r = *rp;
    r.state = 3;
    S.free_slots.push_back(r.slot);
    S.lat.add(t - r.arrival_ns);
    S.lag.add(r.enter_ns - r.arrival_ns);
    S.upload.add(r.admit_ns - r.enter_ns);
    S.queue_wait.add(r.launch_ns - r.admit_ns);
    S.service.add(t - r.launch_ns);
  }
  L.reqs.clear();
  L.busy = false;
}

// The worker owns the lanes. It takes the queue's lock only for host work
// (retiring a finished batch, taking the next batch's tickets); every CUDA
// call (event query, slot-list copy, graph launch) runs without it, so a
// submission never waits behind the driver.
void worker_main(Server* S) {
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(S->I->device);
  while (!S->stop) {
    bool finished[kLanes] = {};
    bool any_busy = false;
    for (int l = 0; l < kLanes; ++l) {
      Lane& L = S->lanes[l];
      if (!L.busy) continue;
      const cudaError_t e = cudaEventQuery(L.done);
      if (e == cudaSuccess) {
        finished[l] = true;
        fill_results(*S, L);
      } else if (e != cudaErrorNotReady) {
        S->worker_error = HNTL_ECUDA;
        S->stop = true;
      }
    }
    uint32_t rows_of[kLanes] = {}, n_of[kLanes] = {};
    size_t graph_of[kLanes] = {};
    bool progressed = false;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (int l = 0; l < kLanes; ++l) {
        Lane& L = S->lanes[l];
        if (finished[l]) {
          retire(*S, L);
          progressed = true;
        }
        if (S->stop || L.busy || S->queue.empty()) continue;
        const uint32_t n = (uint32_t)std::min<size_t>(S->B, S->queue.size());
        size_t gi = 0;
        while (L.graphs[gi].first < n) ++gi;  // the largest graph holds B rows
        const uint32_t rows = L.graphs[gi].first;
        uint32_t first_slot = 0;
        const int64_t t_launch = now_ns();
        for (uint32_t i = 0; i < n; ++i) {
          const uint64_t t = S->queue.front();
          S->queue.pop_front();
          Req& r = S->reqs[t];
          r.state = 2;
          r.launch_ns = t_launch;
          L.h_slots[i] = r.slot;
          if (i == 0) first_slot = r.slot;
          L.reqs.push_back(&r);
        }
        for (uint32_t i = n; i < rows; ++i) L.h_slots[i] = first_slot;  // padding rows, results discarded
        rows_of[l] = rows;
        n_of[l] = n;
        graph_of[l] = gi;
        S->batches += 1;
        S->batched += n;
      }
    }
    if (progressed) S->cv_done.notify_all();
    for (int l = 0; l < kLanes; ++l) {
      Lane& L = S->lanes[l];
      if (!n_of[l]) continue;
      // the lane's previous batch has retired, so its pinned slot list is free to reuse
      if (cudaMemcpyAsync(L.d_slots, L.h_slots, sizeof(uint32_t) * rows_of[l], cudaMemcpyHostToDevice, L.st) !=
              cudaSuccess ||
          cudaGraphLaunch(L.graphs[graph_of[l]].second, L.st) != cudaSuccess ||
          cudaEventRecord(L.done, L.st) != cudaSuccess) {
        // the batch's requests stay unfinished (pollers get the error): the
        // lane's event does not belong to this batch, so nothing may retire
        std::lock_guard<std::mutex> lk(S->mu);
        L.reqs.clear();
        S->worker_error = HNTL_ECUDA;
        S->stop = true;
        break;
      }
      L.busy = true;
      progressed = true;
    }
    for (const Lane& L : S->lanes) any_busy |= L.busy;
    if (progressed || S->stop) continue;
    if (any_busy) {
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    } else {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->queue.empty() && !S->stop) S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
  // drain lanes still on the GPU
  {
    std::lock_guard<std::mutex> lk(S->mu);
    for (Lane& L : S->lanes)
      if (L.busy && cudaEventSynchronize(L.done) == cudaSuccess) {
        fill_results(*S, L);
        retire(*S, L);
      }
  }
  S->cv_done.notify_all();
  if (prev >= 0) cudaSetDevice(prev);
}

void destroy(Server& S) {
  if (S.worker.joinable()) {
    S.stop = true;
    S.cv_work.notify_all();
    S.worker.join();
  }
  for (Lane& L : S.lanes) {
    for (auto& g : L.graphs) cudaGraphExecDestroy(g.second);
    L.graphs.clear();
    if (L.done) cudaEventDestroy(L.done);
    if (L.st) cudaStreamDestroy(L.st);
  }
  for (void* p : S.dev) cudaFree(p);
  for (void* p : S.host) cudaFreeHost(p);
  S.dev.clear();
  S.host.clear();
}

}  // namespace
}  // namespace hntl

struct hntl_server {
  hntl::Server S;
};

using hntl::fail;

extern "C" int hntl_server_create(const hntl_index* idx, size_t mem_budget, uint32_t max_slots, uint32_t batch,
                                  uint32_t nprobe, uint32_t k_max, uint32_t C_max, hntl_server** out) {
  hntl::clear_error();
  if (!idx || !out) return fail(HNTL_EINVAL, "null argument");
  *out = nullptr;
  const hntl::Index& I = idx->I;
  if (batch == 0 || max_slots == 0) return fail(HNTL_EINVAL, "batch and slots must be positive");
  if (!I.X && !I.Xh) return fail(HNTL_EINVAL, "the server reranks raw rows; the index was loaded without them");
  if (C_max < k_max) C_max = k_max;
  const size_t ws = hntl::workspace_bytes(I, batch, k_max, C_max, nprobe);
  if (!ws) return HNTL_EINVAL;
  const size_t lane_bytes = ws + (size_t)batch * (I.d * 4 + 4 + 4 + 4 + 16 + k_max * 12) + 4096;
  if (hntl::kLanes * lane_bytes > mem_budget) return fail(HNTL_ENOMEM, "memory budget below the lanes");
  const uint32_t slots = max_slots;
  hntl_server* h = new (std::nothrow) hntl_server();
  if (!h) return fail(HNTL_ENOMEM, "host allocation");
  hntl::Server& S = h->S;
  S.I = &I;
  S.B = batch;
  S.nprobe = nprobe;
  S.kmax = k_max;
  S.Cmax = C_max;
  S.nslots = slots;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(I.device);
  int rc = HNTL_OK;
  auto dalloc = [&](void** p, size_t bytes) {
    if (rc) return;
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      rc = fail(HNTL_ENOMEM, "server: device allocation");
      return;
    }
    S.dev.push_back(*p);
  };
  auto halloc = [&](void** p, size_t bytes) {
    if (rc) return;
    if (cudaMallocHost(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      rc = fail(HNTL_ENOMEM, "server: pinned allocation");
      return;
    }
    S.host.push_back(*p);
  };
  auto mapped = [&](void** h_p, void** d_p, size_t bytes) {
    if (rc) return;
    if (cudaHostAlloc(h_p, std::max<size_t>(bytes, 16), cudaHostAllocMapped) != cudaSuccess) {
      rc = fail(HNTL_ENOMEM, "server: pinned slot table");
      return;
    }
    S.host.push_back(*h_p);
    if (cudaHostGetDevicePointer(d_p, *h_p, 0) != cudaSuccess) rc = fail(HNTL_ECUDA, "server: slot table mapping");
  };
  mapped((void**)&S.h_slot_q, (void**)&S.d_slot_q, (size_t)slots * I.d * 4);
  mapped((void**)&S.h_slot_k, (void**)&S.d_slot_k, (size_t)slots * 4);
  mapped((void**)&S.h_slot_C, (void**)&S.d_slot_C, (size_t)slots * 4);
  mapped((void**)&S.h_slot_range, (void**)&S.d_slot_range, (size_t)slots * 16);
  for (hntl::Lane& L : S.lanes) {
    dalloc((void**)&L.d_slots, batch * 4);
    dalloc((void**)&L.d_Q, (size_t)batch * I.d * 4);
    dalloc((void**)&L.d_k, batch * 4);
    dalloc((void**)&L.d_C, batch * 4);
    if (I.has_attr) dalloc((void**)&L.d_F, (size_t)batch * 16);
    dalloc((void**)&L.d_ids, (size_t)batch * k_max * 8);
    dalloc((void**)&L.d_dist, (size_t)batch * k_max * 4);
    dalloc(&L.ws, ws);
    L.ws_bytes = ws;
    halloc((void**)&L.h_slots, batch * 4);
    halloc((void**)&L.h_ids, (size_t)batch * k_max * 8);
    halloc((void**)&L.h_dist, (size_t)batch * k_max * 4);
  }
  if (!rc) {
    // neutral slot contents so the warm-up and padding rows are valid requests
    std::memset(S.h_slot_q, 0, (size_t)slots * I.d * 4);
    for (uint32_t i = 0; i < slots; ++i) {
      S.h_slot_k[i] = k_max;
      S.h_slot_C[i] = C_max;
      S.h_slot_range[2 * (size_t)i] = INT64_MIN;
      S.h_slot_range[2 * (size_t)i + 1] = INT64_MAX;
    }
  }
  for (hntl::Lane& L : S.lanes) {
    if (rc) break;
    if (cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess) {
      rc = fail(HNTL_ECUDA, "server: stream/event");
      break;
    }
    cudaMemset(L.d_slots, 0, batch * 4);
    auto record = [&](uint32_t rows) -> int {
      hntl::k_gather_batch<<<rows, 128, 0, L.st>>>(L.d_slots, (int)rows, (int)I.d, S.d_slot_q, S.d_slot_k,
                                                   S.d_slot_C, S.d_slot_range, L.d_Q, L.d_k, L.d_C, L.d_F);
      int r = hntl::search(I, L.d_Q, rows, k_max, C_max, nprobe, L.d_F, L.ws, L.ws_bytes, L.d_ids, L.d_dist,
                           nullptr, nullptr, nullptr, L.st, nullptr, L.d_k, L.d_C, false);
      if (r) return r;
      if (cudaMemcpyAsync(L.h_ids, L.d_ids, (size_t)rows * k_max * 8, cudaMemcpyDeviceToHost, L.st) ||
          cudaMemcpyAsync(L.h_dist, L.d_dist, (size_t)rows * k_max * 4, cudaMemcpyDeviceToHost, L.st))
        return fail(HNTL_ECUDA, "server: result copies");
      return HNTL_OK;
    };
    std::vector<uint32_t> sizes;
    for (uint32_t rows = batch;; rows /= 2) {
      sizes.insert(sizes.begin(), rows);
      if (rows / 2 < 32) break;
    }
    for (uint32_t rows : sizes) {
      // one eager run (sets kernel attributes), then capture the same sequence as a graph
      if ((rc = record(rows))) break;
      if (cudaStreamSynchronize(L.st) != cudaSuccess) {
        rc = fail(HNTL_ECUDA, "server: warm-up batch");
        break;
      }
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(L.st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        rc = fail(HNTL_ECUDA, "server: begin capture");
        break;
      }
      int rr = record(rows);
      cudaError_t ce = cudaStreamEndCapture(L.st, &g);
      if (rr || ce != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        rc = rr ? rr : fail(HNTL_ECUDA, std::string("server: capture: ") + cudaGetErrorString(ce));
        break;
      }
      cudaGraphExec_t ex = nullptr;
      ce = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      if (ce != cudaSuccess) {
        rc = fail(HNTL_ECUDA, std::string("server: instantiate: ") + cudaGetErrorString(ce));
        break;
      }
      L.graphs.emplace_back(rows, ex);
    }
    if (rc) break;
  }
  if (prev >= 0) cudaSetDevice(prev);
  if (rc) {
    hntl::destroy(S);
    delete h;
    return rc;
  }
  for (uint32_t i = slots; i > 0; --i) S.free_slots.push_back(i - 1);
  S.worker = std::thread(hntl::worker_main, &S);
  *out = h;
  return HNTL_OK;
}

extern "C" void hntl_server_free(hntl_server* h) {
  if (!h) return;
  hntl::destroy(h->S);
  delete h;
}

extern "C" int hntl_server_submit(hntl_server* h, const float* h_queries, uint32_t n, const uint32_t* h_k,
                                  const uint32_t* h_C, const int64_t* h_ranges, const int64_t* h_arrival_ns,
                                  uint64_t* tickets, uint32_t* n_admitted) {
  hntl::clear_error();
  if (!h || !n_admitted || (n && (!h_queries || !h_k || !h_C || !tickets))) return fail(HNTL_EINVAL, "null argument");
  hntl::Server& S = h->S;
  *n_admitted = 0;
  const int64_t t_enter = hntl::now_ns();
  if (S.worker_error) return fail(S.worker_error, "the serving worker stopped on a CUDA error");
  if (h_ranges && !S.I->has_attr) return fail(HNTL_EINVAL, "ranges given but the index has no attribute column");
  for (uint32_t i = 0; i < n; ++i)
    if (h_k[i] < 1 || h_k[i] > S.kmax || std::max(h_C[i], h_k[i]) > S.Cmax)
      return fail(HNTL_EINVAL, "k or C beyond the server's k_max / C_max");
  std::unique_lock<std::mutex> lk(S.mu);
  const uint32_t take = (uint32_t)std::min<size_t>(n, S.free_slots.size());
  std::vector<uint32_t> slots(take);
  for (uint32_t i = 0; i < take; ++i) {
    slots[i] = S.free_slots.back();
    S.free_slots.pop_back();
  }
  lk.unlock();
  // rows into their slots with host stores; the slots are this call's alone
  // until it queues them, and the queue's lock orders these stores before the
  // launch of the batch that reads them
  const int64_t t0 = hntl::now_ns();
  const uint32_t d = S.I->d;
  for (uint32_t i = 0; i < take; ++i) {
    const uint32_t s = slots[i];
    std::memcpy(S.h_slot_q + (size_t)s * d, h_queries + (size_t)i * d, (size_t)d * 4);
    S.h_slot_k[s] = h_k[i];
    S.h_slot_C[s] = std::max(h_C[i], h_k[i]);
    S.h_slot_range[2 * (size_t)s] = h_ranges ? h_ranges[2 * (size_t)i] : INT64_MIN;
    S.h_slot_range[2 * (size_t)s + 1] = h_ranges ? h_ranges[2 * (size_t)i + 1] : INT64_MAX;
  }
  lk.lock();
  for (uint32_t i = 0; i < take; ++i) {
    const uint64_t t = S.next_ticket++;
    hntl::Req r;
    r.slot = slots[i];
    r.k = h_k[i];
    r.state = 1;
    r.arrival_ns = h_arrival_ns ? h_arrival_ns[i] : t0;
    r.enter_ns = h_arrival_ns ? t_enter : t0;
    r.admit_ns = hntl::now_ns();
    S.reqs.emplace(t, std::move(r));
    S.queue.push_back(t);
    tickets[i] = t;
  }
  lk.unlock();
  S.cv_work.notify_one();
  *n_admitted = take;
  return take < n ? HNTL_EBUSY : HNTL_OK;
}

extern "C" int hntl_server_poll(hntl_server* h, uint64_t ticket, int64_t* h_ids, float* h_dist, uint32_t timeout_ms) {
  hntl::clear_error();
  if (!h) return fail(HNTL_EINVAL, "null server");
  hntl::Server& S = h->S;
  std::unique_lock<std::mutex> lk(S.mu);
  auto it = S.reqs.find(ticket);
  if (it == S.reqs.end()) return fail(HNTL_EINVAL, "unknown ticket");
  auto finished = [&] {
    auto jt = S.reqs.find(ticket);
    return jt != S.reqs.end() && jt->second.state == 3;
  };
  // wake on the result or on a stopped worker (whose unfinished requests never finish)
  S.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return finished() || S.worker_error != 0; });
  if (!finished()) return S.worker_error ? fail(S.worker_error, "the serving worker stopped") : HNTL_ETIMEOUT;
  hntl::Req& r = S.reqs[ticket];
  if (h_ids) std::copy(r.ids.begin(), r.ids.end(), h_ids);
  if (h_dist) std::copy(r.dist.begin(), r.dist.end(), h_dist);
  S.reqs.erase(ticket);
  return HNTL_OK;
}

extern "C" int hntl_server_poll_many(hntl_server* h, const uint64_t* tickets, uint32_t n, int64_t* h_ids,
                                     float* h_dist, uint32_t stride, uint8_t* done, uint32_t timeout_ms,
                                     uint32_t* n_done) {
  hntl::clear_error();
  if (!h || !n_done || (n && (!tickets || !done))) return fail(HNTL_EINVAL, "null argument");
  hntl::Server& S = h->S;
  *n_done = 0;
  if ((h_ids || h_dist) && stride < S.kmax) return fail(HNTL_EINVAL, "result stride below k_max");
  std::vector<decltype(S.reqs)::node_type> released;  // freed after the lock is dropped
  std::unique_lock<std::mutex> lk(S.mu);
  for (uint32_t i = 0; i < n; ++i)
    if (!done[i] && S.reqs.find(tickets[i]) == S.reqs.end()) return fail(HNTL_EINVAL, "unknown ticket");
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  uint32_t got = 0;
  for (;;) {
    for (uint32_t i = 0; i < n; ++i) {
      if (done[i]) continue;
      auto it = S.reqs.find(tickets[i]);
      if (it == S.reqs.end() || it->second.state != 3) continue;
      hntl::Req& r = it->second;
      if (h_ids) std::copy(r.ids.begin(), r.ids.end(), h_ids + (size_t)i * stride);
      if (h_dist) std::copy(r.dist.begin(), r.dist.end(), h_dist + (size_t)i * stride);
      released.push_back(S.reqs.extract(it));
      done[i] = 1;
      ++got;
    }
    uint32_t left = 0;
    for (uint32_t i = 0; i < n; ++i) left += done[i] ? 0 : 1;
    if (!left) break;
    if (S.worker_error) {
      *n_done = got;
      return fail(S.worker_error, "the serving worker stopped");
    }
    if (S.cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      *n_done = got;
      return HNTL_ETIMEOUT;
    }
  }
  *n_done = got;
  return HNTL_OK;
}

extern "C" int hntl_server_get_stats(hntl_server* h, hntl_server_stats* out) {
  hntl::clear_error();
  if (!h || !out) return fail(HNTL_EINVAL, "null argument");
  hntl::Server& S = h->S;
  std::lock_guard<std::mutex> lk(S.mu);
  out->completed = S.lat.n;
  out->batches = S.batches;
  out->mean_batch = S.batches ? (double)S.batched / (double)S.batches : 0.0;
  out->slots = S.nslots;
  out->p50_us = S.lat.quantile_us(0.50);
  out->p99_us = S.lat.quantile_us(0.99);
  out->max_us = (double)S.lat.max_ns / 1e3;
  out->lag_p50_us = S.lag.quantile_us(0.50);
  out->lag_p99_us = S.lag.quantile_us(0.99);
  out->upload_p50_us = S.upload.quantile_us(0.50);
  out->upload_p99_us = S.upload.quantile_us(0.99);
  out->queue_p50_us = S.queue_wait.quantile_us(0.50);
  out->queue_p99_us = S.queue_wait.quantile_us(0.99);
  out->service_p50_us = S.service.quantile_us(0.50);
  out->service_p99_us = S.service.quantile_us(0.99);
  return HNTL_OK;
}

extern "C" int hntl_server_reset_stats(hntl_server* h) {
  hntl::clear_error();
  if (!h) return fail(HNTL_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(h->S.mu);
  h->S.lat.clear();
  h->S.lag.clear();
  h->S.upload.clear();
  h->S.queue_wait.clear();
  h->S.service.clear();
  h->S.batches = h->S.batched = 0;
  return HNTL_OK;
}

// Open-loop replay: request i goes in at (or right after) its arrival time,
// with the requests that have arrived by then, from this thread; finished
// requests are released every 1 ms (the wanted ones' ids copied out).
extern "C" int hntl_server_replay(hntl_server* h, const float* h_queries, uint32_t n, const uint32_t* h_k,
                                  const uint32_t* h_C, const int64_t* h_ranges, const int64_t* h_arrival_ns,
                                  const uint8_t* h_want, int64_t* h_ids, uint32_t timeout_ms, uint32_t* n_done) {
  hntl::clear_error();
  if (!h || !n_done || (n && (!h_queries || !h_k || !h_C || !h_arrival_ns)) || (h_want && !h_ids))
    return fail(HNTL_EINVAL, "null argument");
  hntl::Server& S = h->S;
  *n_done = 0;
  for (uint32_t i = 1; i < n; ++i)
    if (h_arrival_ns[i] < h_arrival_ns[i - 1]) return fail(HNTL_EINVAL, "replay: arrival times must not decrease");
  const uint32_t d = S.I->d;
  std::vector<uint64_t> tickets(n, 0);
  std::vector<uint8_t> done(n, 0);
  // offsets from the start of the call become steady-clock stamps
  const int64_t t0 = hntl::now_ns();
  std::vector<int64_t> arrival(n);
  for (uint32_t i = 0; i < n; ++i) arrival[i] = t0 + h_arrival_ns[i];
  uint32_t next = 0, lo = 0, finished = 0;
  const int64_t deadline = t0 + (int64_t)timeout_ms * 1000000;
  int64_t last_release = 0;
  std::vector<decltype(S.reqs)::node_type> released;
  auto release = [&]() {
    {
      std::lock_guard<std::mutex> lk(S.mu);
      for (uint32_t i = lo; i < next; ++i) {
        if (done[i]) continue;
        auto it = S.reqs.find(tickets[i]);
        if (it == S.reqs.end() || it->second.state != 3) continue;
        if (h_want && h_want[i])
          std::copy(it->second.ids.begin(), it->second.ids.end(), h_ids + (size_t)i * S.kmax);
        released.push_back(S.reqs.extract(it));
        done[i] = 1;
        ++finished;
      }
    }
    released.clear();  // the entries' memory goes back without the lock held
    while (lo < next && done[lo]) ++lo;
  };
  while (finished < n) {
    const int64_t now = hntl::now_ns();
    if (now > deadline) {
      *n_done = finished;
      return HNTL_ETIMEOUT;
    }
    if (S.worker_error) {
      *n_done = finished;
      return fail(S.worker_error, "the serving worker stopped");
    }
    uint32_t j = next;
    while (j < n && j - next < 4096 && arrival[j] <= now) ++j;
    if (j > next) {
      uint32_t adm = 0;
      const int rc = hntl_server_submit(h, h_queries + (size_t)next * d, j - next, h_k + next, h_C + next,
                                        h_ranges ? h_ranges + 2 * (size_t)next : nullptr, arrival.data() + next,
                                        tickets.data() + next, &adm);
      if (rc != HNTL_OK && rc != HNTL_EBUSY) {
        *n_done = finished;
        return rc;
      }
      next += adm;
    }
    // slots ran out: free the finished ones at once
    if (now - last_release > 1000000 || next == n || next < j) {
      release();
      last_release = now;
    }
    if (next < n && next == j) {  // nothing has arrived yet: wait for the next arrival
      const int64_t wait = std::min(arrival[next], last_release + 1000000) - hntl::now_ns();
      if (wait > 100000) std::this_thread::sleep_for(std::chrono::nanoseconds(wait - 50000));
    } else if (next < j) {  // slots still full after the release
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    } else if (next == n && finished < n) {
      std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
  }
  *n_done = finished;
  return HNTL_OK;
}
