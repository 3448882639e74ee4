// vibe_decode_noalloc: decoding for callers that must not allocate device memory while they decode.
//
// vibe_decode grows a per-handle workspace with cudaMalloc on its first call and whenever a batch
// outgrows it. Some callers cannot allow that: a control loop that must keep a fixed memory
// footprint once it is running, a process that shares the GPU under a hard memory budget, or code
// that runs where the CUDA allocator may not be entered. For them this entry point decodes with
// scratch memory in one file-scope device array of kStaticBytes (64 MiB) per GPU, held until the
// process exits.
//
// When the array comes into being: CUDA loads a library's device code lazily by default (since
// CUDA 12.2, unless CUDA_MODULE_LOADING=EAGER), so the array is placed on a device the first time
// this file's set-up asks for its address -- the first call of this entry point on that device,
// which may therefore need 64 MiB of free device memory. A call with B = 0 does that set-up and
// decodes nothing: make one on each device while allocation is still allowed (and before any
// stream capture); every later call allocates nothing. The address is kept per device for the
// life of the process: after cudaDeviceReset (or anything else that destroys the primary
// context) the entry point must not be used again in that process.
//
// The kernels are the same BP ensemble and LSD kernels vibe_decode runs; only their scratch
// (shot and LSD counters, the LSD hand-off queue, the per-warp LLR accumulators, the per-CTA LSD
// rows) is carved out of the static array instead of the handle's workspace.
#include <cstdio>
#include <mutex>

#include "vibe_internal.cuh"

namespace {

constexpr size_t kStaticBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_lock;
void* g_scratch_addr[kMaxDevices] = {};   // device address of g_static_scratch, per device

// Host code only sees a host-side stand-in for g_static_scratch; the device address comes from
// cudaGetSymbolAddress, resolved once per device with that device current.
int scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return vibe::set_error(VIBE_ERR_UNSUPPORTED, "device index too large");
  std::lock_guard<std::mutex> g(g_lock);
  if (!g_scratch_addr[device]) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != device)
      return vibe::set_error(VIBE_ERR_INVALID, "the handle's device must be current");
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return vibe::set_error(VIBE_ERR_CUDA, cudaGetErrorString(e));
    g_scratch_addr[device] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[device]);
  return VIBE_OK;
}

inline size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" int vibe_decode_noalloc(vibe_handle* h, const uint32_t* d_syndromes, int64_t B, uint32_t* d_corrections,
                                   uint32_t* d_logical, vibe_shot_stats* d_stats, void* stream) {
  vibe::HandleView v;
  int rc = vibe::handle_view(h, &v);
  if (rc != VIBE_OK) return rc;
  if (B < 0) return vibe::set_error(VIBE_ERR_INVALID, "negative batch");
  if (B == 0) {   // set-up only: place the array on this device and look up its address
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != v.device)
      return vibe::set_error(VIBE_ERR_INVALID, "the handle's device must be current");
    unsigned char* base = nullptr;
    return scratch_address(v.device, &base);
  }
  if (!d_syndromes || !d_corrections) return vibe::set_error(VIBE_ERR_INVALID, "NULL syndromes or corrections");
  const vibe::Tables& t = v.t;
  if (t.engine != VIBE_ENGINE_IMAGE)
    return vibe::set_error(VIBE_ERR_UNSUPPORTED, "the static workspace serves warp-engine handles only");
  // Fixed part: counters, two n-float rows per BP warp (LLR accumulator, posterior), one row set per
  // LSD CTA. The LSD CTAs are capped at one per SM so the fixed part stays small; the rest holds the
  // LSD hand-off queue.
  const int bp_grid = v.bp_grid;
  const int lsd_grid = v.lsd_grid < v.num_sms ? v.lsd_grid : v.num_sms;
  const size_t ctrl_b = 256;
  const size_t bp_b = up256((size_t)bp_grid * vibe::kBpWarpsPerCta * 2 * (size_t)t.n * sizeof(float));
  const size_t lsd_b = up256((size_t)lsd_grid * (size_t)vibe::lsd_scratch_words(v.bnd, vibe::kLsdThreads) * sizeof(uint32_t));
  const size_t fixed = ctrl_b + bp_b + lsd_b;
  const size_t per_shot = (size_t)t.n * sizeof(float) + sizeof(uint32_t);
  const long long max_b = fixed + 512 < kStaticBytes ? (long long)((kStaticBytes - fixed - 512) / per_shot) : 0;
  if (B > max_b) {
    char msg[160];
    snprintf(msg, sizeof(msg), "batch of %lld shots exceeds the 64 MiB static workspace (at most %lld for this problem)",
             (long long)B, max_b);
    return vibe::set_error(VIBE_ERR_UNSUPPORTED, msg);
  }
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != v.device)
    return vibe::set_error(VIBE_ERR_INVALID, "the handle's device must be current");
  unsigned char* base = nullptr;
  if ((rc = scratch_address(v.device, &base)) != VIBE_OK) return rc;
  unsigned int* ctrl = reinterpret_cast<unsigned int*>(base);
  float* bp_scratch = reinterpret_cast<float*>(base + ctrl_b);
  uint32_t* lsd_scratch = reinterpret_cast<uint32_t*>(base + ctrl_b + bp_b);
  uint32_t* lsd_shots = reinterpret_cast<uint32_t*>(base + fixed);
  float* lsd_soft = reinterpret_cast<float*>(base + fixed + up256((size_t)B * sizeof(uint32_t)));
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // the array keeps the previous call's contents: the counters must start at zero
  cudaError_t e = cudaMemsetAsync(ctrl, 0, ctrl_b, s);
  if (e != cudaSuccess) return vibe::set_error(VIBE_ERR_CUDA, cudaGetErrorString(e));
  vibe::BpArgs a{};
  a.one = t;
  a.dems = v.d_desc; a.ndem = 1; a.dem_of_shot = nullptr; a.bnd = v.bnd; a.want_soft = 0;
  a.syn = d_syndromes; a.syn_stride = t.mw; a.nshots = (uint32_t)B;
  a.corr = d_corrections; a.corr_stride = t.nw; a.logical = d_logical; a.log_stride = t.kw; a.stats = d_stats;
  a.soft = nullptr; a.soft_stride = t.n; a.obs = nullptr; a.counters = nullptr;
  a.next_shot = ctrl; a.lsd_count = ctrl + 1; a.lsd_shots = lsd_shots; a.lsd_soft = lsd_soft;
  a.scratch = bp_scratch;
  a.scratch_pitch = 2LL * t.n;
  const long long need_ctas = (B + vibe::kBpWarpsPerCta - 1) / vibe::kBpWarpsPerCta;
  const int grid = (int)(need_ctas < bp_grid ? need_ctas : bp_grid);
  if ((e = vibe::launch_bp(a, v.msg_fp16, grid, s)) != cudaSuccess) return vibe::set_error(VIBE_ERR_CUDA, cudaGetErrorString(e));
  vibe::LsdArgs l{};
  l.dems = v.d_desc; l.ndem = 1; l.dem_of_shot = nullptr; l.bnd = v.bnd; l.want_soft = 0;
  l.syn = d_syndromes; l.syn_stride = t.mw; l.corr = d_corrections; l.corr_stride = t.nw;
  l.logical = d_logical; l.log_stride = t.kw; l.stats = d_stats; l.soft = nullptr; l.soft_stride = t.n;
  l.obs = nullptr; l.counters = nullptr;
  l.lsd_count = ctrl + 1; l.lsd_shots = lsd_shots; l.lsd_soft = lsd_soft; l.lsd_next = ctrl + 2;
  l.scratch = lsd_scratch;
  l.scratch_pitch = vibe::lsd_scratch_words(v.bnd, vibe::kLsdThreads);
  if ((e = vibe::launch_lsd(l, lsd_grid, vibe::kLsdThreads, s)) != cudaSuccess) return vibe::set_error(VIBE_ERR_CUDA, cudaGetErrorString(e));
  return VIBE_OK;
}
