// ipm_merge_inplace_noalloc: the plain in-place merge for callers that cannot allocate.
//
// ipm_merge_inplace needs a few megabytes of device scratch (a status block, the split
// table and the exchange plans) that its caller allocates and passes in.  Some callers
// cannot call cudaMalloc at all: code that runs while another framework has reserved
// nearly all device memory for its own pool (a cudaMalloc there fails or forces that
// pool to shrink), latency-critical paths where an allocation, and the device-wide
// synchronisation a later cudaFree implies, is not acceptable, and plain C callers that
// have no allocator of their own to borrow from.  For them this entry point takes the
// scratch from one fixed array compiled into the library instead.
//
// The array is a file-scope __device__ variable, so every GPU that loads the library
// holds it (kScratchBytes) until the process exits.  In host code its name is only a
// host-side stand-in, never a device address: the real address is looked up once per
// device with cudaGetSymbolAddress, with that device current, and passed to the
// kernels as the workspace pointer.
#include <mutex>

#include "ipm_internal.h"

namespace {

// Largest pair count the fixed scratch serves: P = 2^15 pairs, i.e. up to
// 2^15 * 33,792 (~1.1e9) 4-byte keys or 2^15 * 16,896 (~5.5e8) 8-byte keys per call.
// The workspace of such a call (sized for the fused path's split table one level
// deeper, 2^16 + 1 entries, and the exchange plans with their per-section ticket
// prefixes) is ~6.9 MiB for either key width.
constexpr uint32_t kMaxLog2Pairs = 15;
constexpr size_t kScratchBytes = size_t(8) << 20;  // 8 MiB

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// The caller's buffer must be memory of the current device and the stream a stream of
// that device: the array's address differs from device to device and is looked up with
// the current one, so a buffer on another GPU would be handed the wrong GPU's scratch.
// Nothing is launched when this fails.
ipm_status check_current_device(const void *d_buf, cudaStream_t stream, int *dev_out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return IPM_ERR_CUDA;
    }
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, d_buf) != cudaSuccess) {
        (void)cudaGetLastError();
        return IPM_ERR_DEVICE;
    }
    if ((attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) ||
        attr.device != dev)
        return IPM_ERR_DEVICE;
    if (stream != nullptr) {  // the legacy default stream is the current device's
        int sdev = -1;
        if (cudaStreamGetDevice(stream, &sdev) != cudaSuccess) {
            (void)cudaGetLastError();
            return IPM_ERR_CUDA;
        }
        if (sdev != dev) return IPM_ERR_DEVICE;
    }
    *dev_out = dev;
    return IPM_OK;
}

// Device address of g_scratch on device `dev`, the current one (looked up once per
// device).
ipm_status scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) return IPM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_scratch_addr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
            (void)cudaGetLastError();
            return IPM_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return IPM_OK;
}

}  // namespace

extern "C" ipm_status ipm_merge_inplace_noalloc(void *d_buf, uint64_t len_a, uint64_t len_b,
                                                ipm_dtype key_dtype, ipm_stream_t stream) {
    // Size checks first: they need no device and reject what the fixed scratch
    // cannot hold before anything is launched.
    uint32_t G = 0;
    uint64_t tile = 0;
    IPM_TRY(ipm_merge_plan(len_a, len_b, key_dtype, 0, &G, &tile));
    if (G > kMaxLog2Pairs) return IPM_ERR_INVALID_ARG;
    size_t need = 0;
    IPM_TRY(ipm_merge_workspace_bytes(len_a, len_b, key_dtype, 0, 0, &need));
    if (need > kScratchBytes) return IPM_ERR_INVALID_ARG;
    if (len_a + len_b == 0) return IPM_OK;
    if (d_buf == nullptr) return IPM_ERR_INVALID_ARG;
    int dev = 0;
    IPM_TRY(check_current_device(d_buf, (cudaStream_t)stream, &dev));
    void *scratch = nullptr;
    IPM_TRY(scratch_address(dev, &scratch));
    // The merge resets the status block it needs zeroed at the start of every call
    // and writes the split table and plans before reading them, so the previous
    // call's contents of the array do no harm.
    return ipm_merge_inplace(d_buf, len_a, len_b, key_dtype, 0, scratch, kScratchBytes,
                             stream);
}

extern "C" ipm_status ipm_read_noalloc_status(ipm_stream_t stream, ipm_status *out) {
    if (out == nullptr) return IPM_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return IPM_ERR_CUDA;
    }
    void *scratch = nullptr;
    IPM_TRY(scratch_address(dev, &scratch));
    // the array starts with the status block of the last no-alloc call on this device
    return ipm_read_device_status(scratch, stream, out);
}
