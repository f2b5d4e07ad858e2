// d3gb_noalloc.cu -- per-structure energy sums for callers that cannot allocate.
//
// Some callers cannot call cudaMalloc: host programs that keep all device
// memory in their own pool and hand a library only the buffers they own, and
// time-critical loops that cannot afford the implicit device synchronisation
// an allocation may cause.  d3_structure_energies_noalloc gives them the
// per-structure reduction of site energies with no allocation at all: its
// scratch (a copy of the offsets, one partial sum per chunk of atoms, and one
// completion counter per structure) lives in the file-scope array below, which
// every GPU that loads the library holds until the process exits.
//
// Host code cannot use the array's name as a device address; the address is
// looked up once per device with cudaGetSymbolAddress (that device current) on
// the first call there, and kept for the life of the process (calls after a
// cudaDeviceReset are not supported).  Make the first call on a device before
// any stream capture.
//
// The scratch is shared by every call: two calls that overlap on the GPU race
// on it.  Calls on one stream (or otherwise ordered) are safe; the counters
// are cleared by each call before its kernel runs, and everything else is
// overwritten before it is read.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/d3gb.h"

namespace {

constexpr int kChunk = 4096;                // atoms per partial sum
constexpr int kMaxStructs = 16384;          // structures per call
constexpr int kMaxPartials = 65536;         // chunk partial sums per call (structures x chunks)
// layout: offsets int64[kMaxStructs + 1] | partial f64[kMaxPartials] | done u32[kMaxStructs]
constexpr size_t kOffBytes = sizeof(long long) * (kMaxStructs + 1);
constexpr size_t kPartOff = (kOffBytes + 255) / 256 * 256;
constexpr size_t kDoneOff = kPartOff + sizeof(double) * kMaxPartials;
constexpr size_t kScratchBytes = kDoneOff + sizeof(unsigned) * kMaxStructs;  // about 0.7 MB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
d3_status scratch_address(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return D3_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return D3_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_addr[dev]);
    return D3_OK;
}

// Block (c, s) sums the site energies of chunk c of structure s into a partial
// (chunks on grid x, which has no 65535 limit; structures, at most 16384, on
// y); the last block of a structure to finish adds the partials in chunk order.
__global__ void __launch_bounds__(256) k_energy_sums(const long long* __restrict__ off, int maxch,
                                                     const double* __restrict__ e_atom, double* __restrict__ E,
                                                     double* __restrict__ part, unsigned* __restrict__ done) {
    const int ch = blockIdx.x, s = blockIdx.y;
    const long long b = off[s], n = off[s + 1] - b;
    const int nch = (int)((n + kChunk - 1) / kChunk);
    if (n == 0) {
        if (ch == 0 && threadIdx.x == 0) E[s] = 0.0;
        return;
    }
    if (ch >= nch) return;
    const long long k0 = (long long)ch * kChunk, k1 = k0 + kChunk < n ? k0 + kChunk : n;
    double acc = 0.0;
    for (long long k = k0 + threadIdx.x; k < k1; k += blockDim.x) acc += e_atom[b + k];
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    __shared__ bool last;
    if (threadIdx.x == 0) {
        part[(long long)s * maxch + ch] = red[0];
        __threadfence();
        last = atomicAdd(&done[s], 1u) == (unsigned)(nch - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double sum = 0.0;
        for (int c = 0; c < nch; ++c) sum += part[(long long)s * maxch + c];
        E[s] = sum;
    }
}

}  // namespace

extern "C" d3_status d3_structure_energies_noalloc(int32_t B, const int64_t* offsets, const double* e_atom,
                                                   double* E, void* stream) {
    if (B < 0 || !offsets || (B > 0 && !E)) return D3_ERR_ARG;
    if (B == 0) return D3_OK;
    if (B > kMaxStructs) return D3_ERR_CAPACITY;
    if (offsets[0] != 0) return D3_ERR_ARG;
    long long maxn = 0;
    for (int s = 0; s < B; ++s) {
        const long long n = offsets[s + 1] - offsets[s];
        if (n < 0) return D3_ERR_ARG;
        if (n > maxn) maxn = n;
    }
    if (offsets[B] > 0 && !e_atom) return D3_ERR_ARG;
    const long long maxch = maxn > 0 ? (maxn + kChunk - 1) / kChunk : 1;
    if ((long long)B * maxch > kMaxPartials) return D3_ERR_CAPACITY;
    unsigned char* base = nullptr;
    d3_status st = scratch_address(&base);
    if (st != D3_OK) return st;
    long long* off = reinterpret_cast<long long*>(base);
    double* part = reinterpret_cast<double*>(base + kPartOff);
    unsigned* done = reinterpret_cast<unsigned*>(base + kDoneOff);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(off, offsets, sizeof(long long) * (B + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(done, 0, sizeof(unsigned) * B, s);
    if (e != cudaSuccess) return D3_ERR_CUDA;
    k_energy_sums<<<dim3((unsigned)maxch, (unsigned)B), 256, 0, s>>>(off, (int)maxch, e_atom, E, part, done);
    return cudaGetLastError() == cudaSuccess ? D3_OK : D3_ERR_CUDA;
}
