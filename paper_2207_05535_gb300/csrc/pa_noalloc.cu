// Weighted averages that allocate no device memory.
//
// pa_weighted_average copies host records to the device and allocates its
// scratch with cudaMalloc on every call.  Some callers cannot do that:
//  - serving loops that reserve all device memory up front and must not enter
//    the driver's allocator in the steady state (cudaMalloc may synchronise
//    the whole device and stall the other streams),
//  - processes whose device memory is owned by another allocator (a framework
//    caching allocator or a pre-sized arena), where extra cudaMalloc calls
//    compete with it for memory.
// pa_weighted_average_noalloc takes the records and the output already in
// device memory and keeps its scratch (per-run record offsets and the weights
// [n_steps][M]) in the fixed array below, which every GPU that loads this
// library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "pa_internal.cuh"

namespace {

constexpr size_t OFF_BYTES = sizeof(unsigned long long) * PA_NOALLOC_MAX_RUNS;
constexpr size_t W_BYTES = sizeof(double) * PA_NOALLOC_MAX_WEIGHTS;
constexpr size_t SCRATCH_BYTES = OFF_BYTES + W_BYTES;  // 32 KiB + 512 KiB

// Shared by every call on a device; it keeps whatever the last call wrote.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_addr[MAX_DEVICES] = {};

// Device address of the scratch array for the current device.  In host code
// the array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress, looked up once per device with that device current
// and kept for the life of the process (a cudaDeviceReset makes it stale).
pa_status scratch_address(void **out)
{
    int dev = -1;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        std::fprintf(stderr, "libpa: pa_weighted_average_noalloc: no usable current device (%s)\n",
                     cudaGetErrorString(err));
        return PA_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (err != cudaSuccess || !p) {
            std::fprintf(stderr, "libpa: cudaGetSymbolAddress(scratch) failed on device %d: %s\n", dev,
                         cudaGetErrorString(err));
            return PA_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return PA_OK;
}

// Records are contiguous [M][n_steps]: run m starts at record m * n_steps.
__global__ void fill_record_offsets(unsigned long long *off, uint32_t M, uint32_t n_steps)
{
    const uint32_t m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < M) off[m] = (unsigned long long)m * n_steps;
}

}  // namespace

extern "C" pa_status pa_weighted_average_noalloc(const pa_step_record *d_recs, uint32_t M, uint32_t n_steps,
                                                 uint32_t N, uint32_t weight_kind, pa_wavg *d_out,
                                                 void *cuda_stream)
{
    if (!d_recs || !d_out || M == 0 || n_steps == 0 || N == 0 || weight_kind > PA_WEIGHT_SIMPLE)
        return PA_ERR_INVALID_ARG;
    if (M > PA_NOALLOC_MAX_RUNS || (unsigned long long)M * n_steps > PA_NOALLOC_MAX_WEIGHTS) {
        std::fprintf(stderr,
                     "libpa: pa_weighted_average_noalloc: M = %u runs x %u steps exceeds the fixed scratch "
                     "(at most %u runs and %u run-steps)\n",
                     M, n_steps, (unsigned)PA_NOALLOC_MAX_RUNS, (unsigned)PA_NOALLOC_MAX_WEIGHTS);
        return PA_ERR_INVALID_ARG;
    }
    void *base = nullptr;
    pa_status s = scratch_address(&base);
    if (s != PA_OK) return s;
    auto *off = static_cast<unsigned long long *>(base);
    auto *w = reinterpret_cast<double *>(static_cast<unsigned char *>(base) + OFF_BYTES);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // Both scratch regions are written in full by this call before they are
    // read (offsets here, every weight by the averaging kernel), so stale
    // contents from an earlier call are never used.
    fill_record_offsets<<<(M + 255) / 256, 256, 0, st>>>(off, M, n_steps);
    pa::launch_wavg(d_recs, off, nullptr, nullptr, nullptr, 1, M, n_steps, N, weight_kind, d_out, w, nullptr,
                    nullptr, st);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
        std::fprintf(stderr, "libpa: pa_weighted_average_noalloc launch: %s\n", cudaGetErrorString(err));
        return PA_ERR_CUDA;
    }
    return PA_OK;
}
