// pcf_static.cu -- batched sort of small arrays that allocates nothing.
//
// The context entry points size their workspace on demand (cudaMalloc on
// first use or growth, cudaFree on growth and destroy).  Some callers cannot
// allow that: cudaMalloc/cudaFree synchronise the whole device, stalling
// every other stream of the process (a serving loop that keeps several
// streams busy pays that stall on each growth), and a process whose device
// memory is held by a caching allocator or reserved up front by an engine may
// have no memory left to give.  For those callers this entry point runs the
// on-chip path of the library (every array short enough to be finished in
// shared memory, Algorithm 1 with the Sec. 3.3 model run by one warp) with
// all of its scratch in one file-scope device array of fixed size.  It calls no allocating CUDA or library function.
//
// All calls on a device share that array: two calls in flight at the same
// time on one device (two streams, two host threads) race on it and their
// results are undefined; the caller serialises them.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "pcf_internal.h"
#include "pcfsort.h"

namespace pcf {
namespace {

// Fixed limits (the header repeats them as PCF_STATIC_*).
constexpr uint32_t kStCap = 1024;           // keys per array
constexpr uint32_t kStMaxSegs = 65536;      // arrays per call
constexpr uint64_t kStMaxKeys = 1ull << 22; // keys per call

// Layout of the scratch array.
constexpr size_t kOffBrec = 0;                                      // BRec[kStMaxSegs]
constexpr size_t kOffLists = (kOffBrec + sizeof(BRec) * kStMaxSegs + 255) & ~(size_t)255;  // u32[3 S]
constexpr size_t kOffPtab = (kOffLists + 12 * (size_t)kStMaxSegs + 255) & ~(size_t)255;  // u16[4 (cap+1)]
constexpr size_t kOffStatus = (kOffPtab + 8 * (kStCap + 1) + 255) & ~(size_t)255;  // u32[64]: status, class counts
constexpr size_t kStBytes = kOffStatus + 256;

// Extra status bit of this entry point: an offset check failed on the device.
constexpr uint32_t kStBadOffsets = 0x100u;

static __device__ __align__(256) unsigned char g_static_scratch[kStBytes];

// Scratch address of each device (cudaGetSymbolAddress), kept once it was
// resolved; a failed lookup is not kept, so a later call tries again.  A
// device reset (cudaDeviceReset) makes a kept address stale: after one, the
// process must not call this entry point on that device again.
constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void* g_addr[kMaxDevices];

// One thread per array: checks its offsets and writes its record (the
// caller's array s is Learned-Sort at depth 0 with seed + s); one thread per
// size n <= cap: alpha..delta of n; a grid-stride pass over the keys flags
// NaN (binary64 keys).
__global__ void k_static_prepare(const uint64_t* __restrict__ offs, uint32_t S, uint64_t n_total,
                                 uint64_t seed, Policy P, const uint64_t* __restrict__ keys,
                                 uint32_t check_nan, BRec* brec, uint16_t* ptab,
                                 uint32_t* status) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  if (tid < S) {
    const uint64_t a = offs[tid], b = offs[tid + 1];
    const bool bad = b < a || b - a > kStCap || b > n_total || (tid == 0 && a != 0) ||
                     (tid + 1 == S && b != n_total);
    BRec r;
    r.off = (uint32_t)a;
    r.n = bad ? 0u : (uint32_t)(b - a);
    r.kind = (bad || r.n == 0) ? 0u : (BK_LEAF | (r.n < P.tau ? BK_STD : 0u));
    r.depth = 0;
    r.start = 0;
    r.seed = seed + tid;
    brec[tid] = r;
    if (bad) atomicOr(status, kStBadOffsets);
  }
  if (tid <= kStCap) {
    const Params pr = params_of(P, tid);
    ushort4 q;
    q.x = (uint16_t)pr.alpha;
    q.y = (uint16_t)pr.beta;
    q.z = (uint16_t)pr.gamma;
    q.w = (uint16_t)pr.delta;
    if (tid < 2) q = make_ushort4(0, 0, 0, 0);
    reinterpret_cast<ushort4*>(ptab)[tid] = q;
  }
  if (check_nan) {
    bool nan = false;
    for (uint64_t i = tid; i < n_total; i += nthreads) nan |= is_nan_bits(keys[i]);
    if (__any_sync(~0u, nan) && (threadIdx.x & 31) == 0) atomicOr(status, STATUS_NAN);
  }
}

}  // namespace
}  // namespace pcf

using namespace pcf;

extern "C" pcf_status pcf_sort_segmented_static(const void* d_keys_in, void* d_keys_out,
                                                const uint64_t* d_offsets, uint32_t S,
                                                uint64_t n_total, pcf_key_type kt, uint64_t seed,
                                                void* stream) {
  if (kt != PCF_KEY_F64 && kt != PCF_KEY_U64) return PCF_ERR_INVALID_ARG;
  if (S == 0) return n_total == 0 ? PCF_OK : PCF_ERR_INVALID_ARG;
  if (S > kStMaxSegs || n_total > kStMaxKeys) return PCF_ERR_INVALID_ARG;
  if (!d_offsets || (n_total && (!d_keys_in || !d_keys_out))) return PCF_ERR_INVALID_ARG;
  if (((uintptr_t)d_keys_in & 7) || ((uintptr_t)d_keys_out & 7) || ((uintptr_t)d_offsets & 7))
    return PCF_ERR_INVALID_ARG;
  {
    const char* x = (const char*)d_keys_in;
    const char* y = (const char*)d_keys_out;
    if (x != y && x < y + n_total * 8 && y < x + n_total * 8) return PCF_ERR_INVALID_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PCF_ERR_CUDA;
  // the stream must belong to the current device (the scratch is per device)
  {
    int sdev = -1;
    if (cudaStreamGetDevice((cudaStream_t)stream, &sdev) != cudaSuccess) return PCF_ERR_CUDA;
    if (sdev != dev) return PCF_ERR_INVALID_ARG;
  }
  // first call on a device: resolve the scratch address (before any stream
  // capture on that device)
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
      void* a = nullptr;
      if (cudaGetSymbolAddress(&a, g_static_scratch) != cudaSuccess || !a) {
        cudaGetLastError();
        return PCF_ERR_CUDA;
      }
      g_addr[dev] = a;
    }
    base = (unsigned char*)g_addr[dev];
  }
  BRec* brec = (BRec*)(base + kOffBrec);
  uint16_t* ptab = (uint16_t*)(base + kOffPtab);
  uint32_t* status = (uint32_t*)(base + kOffStatus);
  uint32_t* lists = (uint32_t*)(base + kOffLists);
  cudaStream_t st = (cudaStream_t)stream;
  const Policy P{3, 3, 3, 3, 4, MODEL_PCF, 100, RANGE_ARRAY, 0};  // the default policy (Sec. 4)

  // the status word (and, for checked builds, the key limit after it: zero,
  // no limit) is the only scratch that must start at zero here (the
  // class counts are cleared by the on-chip launch itself); the records,
  // lists and table are fully written before they are read
  if (cudaMemsetAsync(status, 0, 16, st) != cudaSuccess) return PCF_ERR_CUDA;
  const uint64_t work = std::max<uint64_t>(std::max<uint64_t>(S, kStCap + 1), n_total / 8);
  const uint32_t grid = (uint32_t)std::min<uint64_t>((work + 255) / 256, 1024);
  k_static_prepare<<<grid, 256, 0, st>>>(d_offsets, S, n_total, seed, P,
                                         (const uint64_t*)d_keys_in, kt == PCF_KEY_F64 ? 1u : 0u,
                                         brec, ptab, status);
  if (cudaGetLastError() != cudaSuccess) return PCF_ERR_CUDA;  // nothing was launched
  uint32_t h_status = 0;
  if (cudaMemcpyAsync(&h_status, status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PCF_ERR_CUDA;
  if (h_status & kStBadOffsets) return PCF_ERR_INVALID_ARG;
  if (h_status & STATUS_NAN) return PCF_ERR_INVALID_KEY;
  if (n_total == 0) return PCF_OK;

  LaunchCfg lc;
  lc.stream = st;
  lc.kt = (uint32_t)kt;
  lc.pairs = false;
  lc.status = status;
  lc.launches = nullptr;
  if (launch_onchip(lc, brec, S, kStCap, (const uint64_t*)d_keys_in, nullptr,
                    (uint64_t*)d_keys_out, nullptr, P, ptab, lists, status + 16) != cudaSuccess) {
    cudaStreamSynchronize(st);  // return with none of this call's work in flight
    return PCF_ERR_CUDA;
  }
  if (cudaMemcpyAsync(&h_status, status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PCF_ERR_CUDA;
  if (h_status & STATUS_TIMEOUT) return PCF_ERR_TIMEOUT;
  if (h_status & (STATUS_INTERNAL | STATUS_BOUNDS)) return PCF_ERR_INTERNAL;
  return PCF_OK;
}
