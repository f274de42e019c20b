// gks_noalloc.cu -- gks_diagnostics_noalloc: the FP64 mass / momentum /
// kinetic-energy reduction for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: a host application that owns
// every byte of device memory through its own pool and forbids libraries to
// allocate behind its back, a process whose device-memory budget is fixed
// and fully committed, or a loop with hard timing bounds where an allocation
// (and a possible failure of it) is not acceptable. This entry point keeps
// its scratch -- one partial sum per block -- in a file-scope static device
// array of fixed size, so it allocates nothing; the caller still passes the
// input state and the output buffer.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "gks_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 16;
constexpr long kCellsPerBlock = (long)kThreads * kCellsPerThread;   // 4096
constexpr int kMaxBlocks = 8192;
constexpr long kMaxCells = kCellsPerBlock * kMaxBlocks;              // 33,554,432
constexpr int kMaxDevices = 64;

// Scratch of every call: 8 doubles per block (5 used), 512 KiB. Every GPU
// that loads the library holds it until the process exits.
static __device__ __align__(256) double g_partials[kMaxBlocks * 8];

std::mutex g_mu;
double *g_scratch[kMaxDevices] = {};

// Device address of g_partials on the current device. In host code the
// symbol name is only a host-side stand-in, so the address is looked up with
// that device current. A call outside stream capture looks it up again every
// time (cheap once the module is loaded), so a device reset or a re-created
// primary context, which reload the module at another address, never leaves
// a stale pointer behind; a call inside a capture cannot make that query and
// takes the address of the last uncaptured call on the device.
int scratch_address(cudaStream_t stream, double **out, std::string *msg)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { *msg = std::string("cudaGetDevice: ") + cudaGetErrorString(e); return GKS_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) { *msg = "device ordinal out of range"; return GKS_ERR_ARG; }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) { *msg = std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e); return GKS_ERR_CUDA; }
    std::lock_guard<std::mutex> lock(g_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_partials);
        if (e != cudaSuccess || !p) {
            *msg = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return GKS_ERR_CUDA;
        }
        g_scratch[dev] = p;
    } else if (!g_scratch[dev]) {
        *msg = "the first call on a device must come before any stream capture";
        return GKS_ERR_STATE;
    }
    *out = g_scratch[dev];
    return GKS_OK;
}

// Block b sums cells [b*4096, (b+1)*4096): thread t takes the cells
// b*4096 + t + 256 k, k = 0..15, then a fixed shared-memory tree. Every
// partial that the final pass reads is written here by the same call, so
// nothing in the scratch has to start at zero.
__global__ void __launch_bounds__(kThreads) noalloc_partial_kernel(const double *q, long N, int nx, int ny,
                                                                    const double *hx, const double *hy,
                                                                    const double *hz, double *partials)
{
    __shared__ double sh[5][kThreads];
    double s[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < kCellsPerThread; ++k) {
        const long c = (long)blockIdx.x * kCellsPerBlock + threadIdx.x + (long)k * kThreads;
        if (c >= N) break;
        const int i = (int)(c % nx);
        const long r = c / nx;
        const int j = (int)(r % ny), kk = (int)(r / ny);
        const double vol = hx[i] * hy[j] * hz[kk];
        const double rho = q[c], mx = q[N + c], my = q[2 * N + c], mz = q[3 * N + c];
        s[0] += rho * vol;
        s[1] += mx * vol;
        s[2] += my * vol;
        s[3] += mz * vol;
        s[4] += 0.5 * (mx * mx + my * my + mz * mz) / rho * vol;
    }
    for (int v = 0; v < 5; ++v) sh[v][threadIdx.x] = s[v];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int v = 0; v < 5; ++v) sh[v][threadIdx.x] += sh[v][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 5) partials[blockIdx.x * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kThreads) noalloc_final_kernel(const double *partials, int nblocks, double *out)
{
    __shared__ double sh[5][kThreads];
    double s[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += kThreads)
        for (int v = 0; v < 5; ++v) s[v] += partials[b * 8 + v];
    for (int v = 0; v < 5; ++v) sh[v][threadIdx.x] = s[v];
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int v = 0; v < 5; ++v) sh[v][threadIdx.x] += sh[v][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 5) out[threadIdx.x] = sh[threadIdx.x][0];
}

}  // namespace

extern "C" int gks_diagnostics_noalloc(const double *d_state, int nx, int ny, int nz, const double *d_hx,
                                       const double *d_hy, const double *d_hz, double *d_out, void *stream)
{
    std::string msg;
    if (!d_state || !d_hx || !d_hy || !d_hz || !d_out) {
        gks::record_error("gks_diagnostics_noalloc: null pointer");
        return GKS_ERR_ARG;
    }
    if (nx < 1 || ny < 1 || nz < 1) {
        gks::record_error("gks_diagnostics_noalloc: every extent must be >= 1");
        return GKS_ERR_ARG;
    }
    const long N = (long)nx * ny * nz;
    if (N > kMaxCells) {
        gks::record_error("gks_diagnostics_noalloc: at most 33554432 cells (static scratch of 8192 blocks "
                          "of 4096 cells); use gks_diagnostics for larger grids");
        return GKS_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    double *scratch = nullptr;
    int rc = scratch_address(s, &scratch, &msg);
    if (rc) {
        gks::record_error(("gks_diagnostics_noalloc: " + msg).c_str());
        return rc;
    }
    const int nblocks = (int)((N + kCellsPerBlock - 1) / kCellsPerBlock);
    noalloc_partial_kernel<<<nblocks, kThreads, 0, s>>>(d_state, N, nx, ny, d_hx, d_hy, d_hz, scratch);
    noalloc_final_kernel<<<1, kThreads, 0, s>>>(scratch, nblocks, d_out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        gks::record_error((std::string("gks_diagnostics_noalloc: ") + cudaGetErrorString(e)).c_str());
        return GKS_ERR_CUDA;
    }
    return GKS_OK;
}
