// ipgc_color_noalloc: the single-graph colouring without any allocation.
//
// Some callers cannot allocate device memory at the moment they want a
// colouring: code running inside a custom allocator or memory-pool callback
// (which must not re-enter the allocator), code holding a fixed memory budget
// that was reserved up front, or a process whose allocator is already
// exhausted but still has room to run a kernel. For them this entry point
// takes its working memory from one file-scope device array of fixed size
// instead of cudaMalloc. Inputs and outputs are still the caller's.
//
// The array below belongs to the library's device code (kScratchBytes =
// 15,074,048 bytes, about 15.1 MB). With lazy module loading (the CUDA
// default) that code, and with it the array, is loaded onto a GPU the first
// time the process uses it there; the first call of this entry point on a
// device looks up the array's address, which loads it if nothing else did.
// That call should therefore be made at set-up, before any stream capture and
// before the moment when allocating is no longer possible; an empty graph
// (n = 0) will do. From then on the device holds the array until the process
// exits. Every call on a device shares that device's copy, which keeps the
// contents of the last call; calls that overlap on one GPU (from different
// streams or host threads) overwrite each other's state, so the caller must
// serialise them. What must start at zero (the control block and the
// validation state) is cleared by every call.
//
// The colouring is the rescanning one of ipgc_color_ex (every round rereads
// the active nodes' rows) with the default degree bound t1 = 64 fixed, the
// default work-item size and threshold rule, without forbidden-colour bitmaps
// or neighbour filtering; its colours, rounds and mode counts are those of
// ipgc_color_ex with default options.
#include <cstring>
#include <mutex>

#include "ipgc_internal.h"

namespace ipgc {
namespace {

// Limits of the fixed scratch (the degree thresholds are the defaults).
constexpr int64_t kNaMaxN = 524288;
constexpr int64_t kNaMaxNnz = 8388608;
constexpr int kNaT1 = kDefaultT1;
constexpr int kNaChunk = kDefaultChunk;

constexpr int64_t al256(int64_t x) { return (x + 255) & ~int64_t(255); }
constexpr int64_t kNaBig = (kNaMaxNnz / (kNaT1 + 1)) < kNaMaxN ? kNaMaxNnz / (kNaT1 + 1) : kNaMaxN;
constexpr int64_t kNaItems = kNaMaxNnz / kNaChunk + kNaBig + 1;
constexpr int64_t kNaGcap = kNaMaxNnz / (kNaChunk + 1) + 1;

// Byte offsets inside the scratch.
constexpr int64_t kOffCtrl = 0;
constexpr int64_t kOffErr = kOffCtrl + al256(sizeof(Ctrl));
constexpr int64_t kOffTent = kOffErr + 256;
constexpr int64_t kOffWl0 = kOffTent + al256(4 * kNaMaxN);
constexpr int64_t kOffWl1 = kOffWl0 + al256(4 * kNaMaxN);
constexpr int64_t kOffItems0 = kOffWl1 + al256(4 * kNaMaxN);
constexpr int64_t kOffItems1 = kOffItems0 + al256(16 * kNaItems);
constexpr int64_t kOffIstat = kOffItems1 + al256(16 * kNaItems);
constexpr int64_t kOffGbits = kOffIstat + al256(16 * kNaItems);
constexpr int64_t kOffDoneA = kOffGbits + al256(4 * kGWords * kNaGcap);
constexpr int64_t kOffDoneD = kOffDoneA + al256(4 * kNaGcap);
constexpr int64_t kOffFlag = kOffDoneD + al256(4 * kNaGcap);
constexpr int64_t kScratchBytes = kOffFlag + al256(4 * kNaGcap);

// The fixed working memory of ipgc_color_noalloc (see the file comment).
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceSetup {
  bool ready = false;
  unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch
  int sms = 0;
  int occ = 0;  // resident CTAs per SM of the colouring kernel (256 threads)
};

constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

// Once per device, with that device current: resolve the array's device
// address (host code cannot use the symbol itself) and the launch shape.
int setup_device(int dev, DeviceSetup* out) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  DeviceSetup& d = g_setup[dev];
  if (!d.ready) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return IPGC_ERR_CUDA;
    int sms = 0, occ = 0, coop = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return IPGC_ERR_CUDA;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess)
      return IPGC_ERR_CUDA;
    if (occupancy_persistent(256, &occ) != cudaSuccess) return IPGC_ERR_CUDA;
    if (!coop || occ < 1) return IPGC_ERR_UNSUPPORTED;
    d.scratch = static_cast<unsigned char*>(ptr);
    d.sms = sms;
    d.occ = occ;
    d.ready = true;
  }
  *out = d;
  return IPGC_OK;
}

}  // namespace
}  // namespace ipgc

extern "C" IPGC_API int ipgc_color_noalloc(const int32_t* rowptr, const int32_t* col, int32_t n,
                                           int64_t nnz, int32_t* colors_out,
                                           ipgc_stats* stats_out, void* stream) {
  using namespace ipgc;
  // arguments and limits are checked before any CUDA call
  if (n < 0 || nnz < 0) return IPGC_ERR_INVALID;
  if (n > kNaMaxN || nnz > kNaMaxNnz) return IPGC_ERR_TOO_LARGE;
  if (n > 0 && (!rowptr || !colors_out)) return IPGC_ERR_INVALID;
  if (nnz > 0 && (!col || n == 0)) return IPGC_ERR_INVALID;
  if (stats_out) std::memset(stats_out, 0, sizeof(*stats_out));

  // the per-device set-up comes first, so that an empty call made at
  // initialisation already reserves the array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return IPGC_ERR_CUDA;
  DeviceSetup ds;
  int rc = setup_device(dev, &ds);
  if (rc != IPGC_OK) return rc;
  if (n == 0) return IPGC_OK;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = ds.scratch;

  // the control block and the validation state must start at zero
  if (cudaMemsetAsync(base, 0, (size_t)kOffTent, s) != cudaSuccess) return IPGC_ERR_CUDA;
  ValidateState* d_err = reinterpret_cast<ValidateState*>(base + kOffErr);
  if (launch_validate(rowptr, col, n, nnz, d_err, ds.sms * 8, s) != cudaSuccess) return IPGC_ERR_CUDA;
  int h_err = 0;
  if (cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return IPGC_ERR_CUDA;
  if (h_err) return IPGC_ERR_INVALID;

  Params p;
  std::memset(&p, 0, sizeof(p));
  p.rowptr = rowptr;
  p.col = col;
  p.n = n;
  p.nnz = nnz;
  p.color = colors_out;
  p.tent = reinterpret_cast<int32_t*>(base + kOffTent);
  p.wl[0] = reinterpret_cast<int32_t*>(base + kOffWl0);
  p.wl[1] = reinterpret_cast<int32_t*>(base + kOffWl1);
  p.items[0] = reinterpret_cast<int4*>(base + kOffItems0);
  p.items[1] = reinterpret_cast<int4*>(base + kOffItems1);
  p.istat = reinterpret_cast<int4*>(base + kOffIstat);
  p.gbits = reinterpret_cast<uint32_t*>(base + kOffGbits);
  p.done_a = reinterpret_cast<int32_t*>(base + kOffDoneA);
  p.done_d = reinterpret_cast<int32_t*>(base + kOffDoneD);
  p.flag = reinterpret_cast<int32_t*>(base + kOffFlag);
  p.ctrl = reinterpret_cast<Ctrl*>(base + kOffCtrl);
  p.t1 = kNaT1;
  p.chunk = kNaChunk;
  p.H = (int64_t)(0.6 * (double)n);
  p.policy = IPGC_MODE_THRESHOLD;
  p.max_rounds = n + 1;
  p.timeout_ns = 10000000000ull;
  p.col_vec = ((uintptr_t)col & 15u) == 0 ? 1 : 0;
  if (launch_persistent(p, 256, ds.occ * ds.sms, 0, s) != cudaSuccess) return IPGC_ERR_CUDA;

  // the call always waits for the colouring, so that an error the device
  // reported (a bounded wait that expired, too many rounds) is returned
  Ctrl h;
  if (cudaMemcpyAsync(&h, p.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return IPGC_ERR_CUDA;
  if (stats_out) {
    stats_out->rounds = h.rounds;
    stats_out->num_colors = h.maxc;
    stats_out->rounds_topo = h.rounds_topo;
    stats_out->rounds_data = h.rounds_data;
    stats_out->edges_processed = (int64_t)h.edges;
    stats_out->ns = h.t_end >= h.t_start ? h.t_end - h.t_start : 0;
    stats_out->error = h.status;
  }
  return h.status;
}
