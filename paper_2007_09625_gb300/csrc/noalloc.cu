// noalloc.cu -- gbsz_codebook_noalloc: the Huffman codebook kernel (S4) for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: host frameworks that own all device
// memory through their own pool and forbid driver allocations behind their
// back, and processes that run under a fixed device-memory budget where a
// library allocating on its own could push them over it.  For them, this
// entry point runs the same codebook kernel as the compressor, with all of
// its scratch in one file-scope device array of fixed size instead of a
// context's allocations.
//
// The array is sized for the largest alphabet the format allows (65536
// symbols) and takes about 4 MB on every GPU that loads this library, until
// the process exits.  Every call shares it and it keeps the last call's
// contents, so two calls whose kernels overlap on the GPU race: serialise
// them (one stream, or events).  The control block is cleared on every call.
// The call reads its status back and synchronises its stream before it
// returns.
#include "../../include/gbsz.h"
#include "common.cuh"

#include <cstring>
#include <mutex>

using namespace gbsz;

namespace {

constexpr size_t kB = kMaxBins;
// byte offsets of the scratch regions inside the array (all 256-aligned)
constexpr size_t kOffCtl = 0;
constexpr size_t kOffKeyA = 256;
constexpr size_t kOffKeyB = kOffKeyA + kB * 8;
constexpr size_t kOffNodeF = kOffKeyB + kB * 8;
constexpr size_t kOffParent = kOffNodeF + kB * 4;
constexpr size_t kOffDistA = kOffParent + 2 * kB * 4;
constexpr size_t kOffDistB = kOffDistA + 2 * kB * 4;
constexpr size_t kOffParA = kOffDistB + 2 * kB * 4;
constexpr size_t kOffParB = kOffParA + 2 * kB * 4;
constexpr size_t kOffCw64 = kOffParB + 2 * kB * 4;
constexpr size_t kOffCw32 = kOffCw64 + kB * 8;
constexpr size_t kScratchBytes = kOffCw32 + kB * 4;
static_assert(sizeof(Control) <= 256, "control block must fit its slot");

__device__ __align__(256) unsigned char g_codebook_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices];  // device address of the array, per device

// Device address of the array on the current device, looked up once per
// device.  The symbol's name in host code is only a host-side stand-in.
gbsz_status scratch_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return GBSZ_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_codebook_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return GBSZ_ERR_CUDA;
        }
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return GBSZ_OK;
}

}  // namespace

extern "C" gbsz_status gbsz_codebook_noalloc(const uint32_t *d_hist, uint32_t nbins, uint8_t *d_len,
                                             uint64_t *d_code, uint32_t *maxlen, void *stream)
{
    if (!d_hist || !d_len || !d_code || nbins < 1 || nbins > kMaxBins) return GBSZ_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GBSZ_ERR_CUDA;
    }
    unsigned char *base = nullptr;
    gbsz_status s = scratch_address(dev, &base);
    if (s != GBSZ_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Control *ctl = reinterpret_cast<Control *>(base + kOffCtl);
    if (cudaMemsetAsync(ctl, 0, sizeof(Control), st) != cudaSuccess) return GBSZ_ERR_CUDA;
    CodebookArgs a{};
    a.hist = d_hist;
    a.nbins = nbins;
    a.len_out = d_len;
    a.codes_only = d_code;
    a.cw64 = reinterpret_cast<uint64_t *>(base + kOffCw64);
    a.cw32 = reinterpret_cast<uint32_t *>(base + kOffCw32);
    a.keyA = reinterpret_cast<unsigned long long *>(base + kOffKeyA);
    a.keyB = reinterpret_cast<unsigned long long *>(base + kOffKeyB);
    a.nodef = reinterpret_cast<uint32_t *>(base + kOffNodeF);
    a.parent = reinterpret_cast<uint32_t *>(base + kOffParent);
    a.distA = reinterpret_cast<uint32_t *>(base + kOffDistA);
    a.distB = reinterpret_cast<uint32_t *>(base + kOffDistB);
    a.parA = reinterpret_cast<uint32_t *>(base + kOffParA);
    a.parB = reinterpret_cast<uint32_t *>(base + kOffParB);
    a.ctl = ctl;
    launch_codebook(a, st);
    if (cudaGetLastError() != cudaSuccess) return GBSZ_ERR_CUDA;
    uint32_t res[2] = {0, 0};  // error bits, maxlen (pageable host copy)
    if (cudaMemcpyAsync(&res[0], &ctl->error, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&res[1], &ctl->maxlen, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return GBSZ_ERR_CUDA;
    if (maxlen) *maxlen = res[1];
    return res[0] ? GBSZ_ERR_INVALID_ARG : GBSZ_OK;
}
