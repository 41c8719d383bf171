// k_noalloc.cu -- solvent observables of caller-owned device arrays, with no
// device allocation.
//
// rmpcd_observables reduces through buffers that rmpcd_create allocated (the
// cell counts of a rebinning pass and per-tile partial sums).  This variant
// takes the solvent as plain device arrays (cell key, velocity, flags), as
// rmpcd_get_state hands them out, and reduces through one file-scope static
// device array instead.  It exists for callers that must not allocate device
// memory at the point where they measure:
//   - a monitor that runs between steps of a simulation whose device memory is
//     wholly reserved by another pool (a framework's caching allocator): an
//     allocation there can fail with out-of-memory;
//   - a caller that keeps work in flight on other streams: cudaFree
//     synchronises the whole device and would stall that work.
//
// The estimator is the §1.4 temperature: per cell with N >= 2,
// 1/(N-1) sum_i |v_i - v_cell|^2, summed over cells and divided by 3 N_c.
// Sums use FP64 atomics, so the last bits depend on the order in which the
// atomics land; results agree with rmpcd_observables to rounding.
//
// The scratch is one array per device (each device that loads this library
// gets its own copy).  Two calls whose work overlaps on one device (different
// streams, or different host threads) share it and race; calls queued on one
// stream run one after another and are safe.

#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <mutex>
#include <string>

#include "rmpcd.h"

namespace rmpcd {
void note_global_error(const std::string &msg);
}

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_DEVICES = 64;
constexpr long long NA_MAX_CELLS = RMPCD_NOALLOC_MAX_CELLS;

// Layout of the scratch (byte offsets, each a multiple of 256):
//   sum[3][NA_MAX_CELLS]  double   per-cell velocity sums
//   dev[NA_MAX_CELLS]     double   per-cell sum of |v - v_cell|^2
//   cnt[NA_MAX_CELLS]     uint32   per-cell particle counts
//   tot[8]                double   totals (see k_na_cells)
//   done                  uint32   blocks of k_na_cells that have finished
// Every field is zeroed by k_na_zero at the start of each call, over the
// first n_cells cells only; nothing is assumed about what a previous call
// left behind.
constexpr size_t NA_OFF_SUM = 0;
constexpr size_t NA_OFF_DEV = NA_OFF_SUM + 3 * NA_MAX_CELLS * sizeof(double);
constexpr size_t NA_OFF_CNT = NA_OFF_DEV + NA_MAX_CELLS * sizeof(double);
constexpr size_t NA_OFF_TOT = NA_OFF_CNT + NA_MAX_CELLS * sizeof(unsigned int);
constexpr size_t NA_OFF_DONE = NA_OFF_TOT + 256;
constexpr size_t NA_SCRATCH_BYTES = NA_OFF_DONE + 256;
static_assert(NA_OFF_DEV % 256 == 0 && NA_OFF_CNT % 256 == 0 && NA_OFF_TOT % 256 == 0, "scratch alignment");

static __device__ __align__(256) unsigned char g_na_scratch[NA_SCRATCH_BYTES];

struct NaView {
    double *sum;          // sum[k * NA_MAX_CELLS + c]
    double *dev;
    unsigned int *cnt;
    double *tot;
    unsigned int *done;
};

NaView view_of(void *base)
{
    unsigned char *b = static_cast<unsigned char *>(base);
    return NaView{reinterpret_cast<double *>(b + NA_OFF_SUM), reinterpret_cast<double *>(b + NA_OFF_DEV),
                  reinterpret_cast<unsigned int *>(b + NA_OFF_CNT), reinterpret_cast<double *>(b + NA_OFF_TOT),
                  reinterpret_cast<unsigned int *>(b + NA_OFF_DONE)};
}

__device__ __forceinline__ double block_sum(double x, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = x;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NA_THREADS / 32; ++w) s += sh[w];
    return s;   // valid on thread 0
}

__global__ void __launch_bounds__(NA_THREADS) k_na_zero(NaView s, int n_cells)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += stride) {
        s.sum[c] = 0.0;
        s.sum[NA_MAX_CELLS + c] = 0.0;
        s.sum[2 * NA_MAX_CELLS + c] = 0.0;
        s.dev[c] = 0.0;
        s.cnt[c] = 0u;
    }
    if (blockIdx.x == 0 && threadIdx.x < 8) s.tot[threadIdx.x] = 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *s.done = 0u;
}

// Pass 1: per-cell count and velocity sums; totals of momentum, kinetic
// energy, species B and particles counted.
__global__ void __launch_bounds__(NA_THREADS) k_na_sums(NaView s, const int *cell, const double *v,
                                                        const unsigned char *flags, long long n, int n_cells)
{
    __shared__ double sh[NA_THREADS / 32];
    double acc[6] = {0, 0, 0, 0, 0, 0};   // px, py, pz, ke, nB, n
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int c = cell[i];
        if (c < 0 || c >= n_cells) continue;
        const double vx = v[3 * i], vy = v[3 * i + 1], vz = v[3 * i + 2];
        atomicAdd(&s.cnt[c], 1u);
        atomicAdd(&s.sum[c], vx);
        atomicAdd(&s.sum[NA_MAX_CELLS + c], vy);
        atomicAdd(&s.sum[2 * NA_MAX_CELLS + c], vz);
        acc[0] += vx;
        acc[1] += vy;
        acc[2] += vz;
        acc[3] += 0.5 * (vx * vx + vy * vy + vz * vz);
        acc[4] += (flags && (flags[i] & 1u)) ? 1.0 : 0.0;
        acc[5] += 1.0;
    }
    for (int k = 0; k < 6; ++k) {
        const double b = block_sum(acc[k], sh);
        if (threadIdx.x == 0 && b != 0.0) atomicAdd(&s.tot[2 + k], b);
    }
}

// Pass 2: per-cell sum of squared deviations from the cell mean.
__global__ void __launch_bounds__(NA_THREADS) k_na_dev(NaView s, const int *cell, const double *v, long long n,
                                                       int n_cells)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int c = cell[i];
        if (c < 0 || c >= n_cells) continue;
        const unsigned int m = s.cnt[c];
        if (m < 2u) continue;
        const double inv = 1.0 / (double)m;
        const double ux = v[3 * i] - s.sum[c] * inv;
        const double uy = v[3 * i + 1] - s.sum[NA_MAX_CELLS + c] * inv;
        const double uz = v[3 * i + 2] - s.sum[2 * NA_MAX_CELLS + c] * inv;
        atomicAdd(&s.dev[c], ux * ux + uy * uy + uz * uz);
    }
}

// Pass 3: per-cell temperature terms, then the last block to finish writes
// out[8] = {T, px, py, pz, kinetic, N_c, N_B, particles counted}.
__global__ void __launch_bounds__(NA_THREADS) k_na_cells(NaView s, int n_cells, double *out)
{
    __shared__ double sh[NA_THREADS / 32];
    __shared__ bool last;
    double t = 0.0, nc = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += stride) {
        const unsigned int m = s.cnt[c];
        if (m >= 2u) {
            t += s.dev[c] / (double)(m - 1u);
            nc += 1.0;
        }
    }
    const double bt = block_sum(t, sh);
    const double bn = block_sum(nc, sh);
    if (threadIdx.x == 0) {
        if (bt != 0.0) atomicAdd(&s.tot[0], bt);
        if (bn != 0.0) atomicAdd(&s.tot[1], bn);
        __threadfence();
        last = atomicAdd(s.done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double tot[8];
        for (int k = 0; k < 8; ++k) tot[k] = __ldcg(&s.tot[k]);
        out[0] = tot[1] > 0.0 ? tot[0] / (3.0 * tot[1]) : 0.0;
        out[1] = tot[2];
        out[2] = tot[3];
        out[3] = tot[4];
        out[4] = tot[5];
        out[5] = tot[1];
        out[6] = tot[6];
        out[7] = tot[7];
    }
}

std::atomic<void *> g_na_ptr[NA_MAX_DEVICES];
std::mutex g_na_mutex;

rmpcd_status na_fail(rmpcd_status st, const char *fmt, long long a = 0, long long b = 0)
{
    char buf[256];
    std::snprintf(buf, sizeof buf, fmt, a, b);
    rmpcd::note_global_error(std::string("rmpcd_observables_noalloc: ") + buf);
    return st;
}

// Resolve this device's scratch address and load the four kernels once per
// device (the caller's current device).  Returns nullptr on failure.
void *na_setup(int dev, cudaError_t *err)
{
    void *p = g_na_ptr[dev].load(std::memory_order_acquire);
    if (p) return p;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    p = g_na_ptr[dev].load(std::memory_order_relaxed);
    if (p) return p;
    cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_na_zero);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_na_sums);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_na_dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_na_cells);
    if (e != cudaSuccess || p == nullptr) {
        *err = e;
        return nullptr;
    }
    g_na_ptr[dev].store(p, std::memory_order_release);
    return p;
}

int grid_for(long long work, int max_blocks)
{
    long long b = (work + NA_THREADS - 1) / NA_THREADS;
    if (b < 1) b = 1;
    return (int)(b < max_blocks ? b : max_blocks);
}

}  // namespace

extern "C" rmpcd_status rmpcd_observables_noalloc(const int32_t *cell, const double *v, const uint8_t *flags,
                                                  int64_t n, int32_t n_cells, double *out, void *stream)
{
    if (n < 0) return na_fail(RMPCD_EINVAL, "n = %lld is negative", (long long)n);
    if (n_cells < 1 || n_cells > NA_MAX_CELLS)
        return na_fail(RMPCD_EINVAL, "n_cells = %lld is outside 1..%lld (the static scratch limit)",
                       (long long)n_cells, NA_MAX_CELLS);
    if (!out) return na_fail(RMPCD_EINVAL, "out is NULL");
    if (n > 0 && (!cell || !v)) return na_fail(RMPCD_EINVAL, "cell or v is NULL with n = %lld", (long long)n);
    if (((uintptr_t)v & 7u) || ((uintptr_t)out & 7u) || ((uintptr_t)cell & 3u))
        return na_fail(RMPCD_EINVAL, "misaligned pointer (v and out need 8 bytes, cell 4 bytes)");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(RMPCD_ECUDA, "cudaGetDevice failed (error %lld)", (long long)e);
    if (dev < 0 || dev >= NA_MAX_DEVICES)
        return na_fail(RMPCD_EINVAL, "device %lld is beyond the %lld devices supported", dev, NA_MAX_DEVICES);
    e = cudaSuccess;
    void *base = na_setup(dev, &e);
    if (!base) return na_fail(RMPCD_ECUDA, "scratch setup failed (CUDA error %lld)", (long long)e);
    int n_sm = 0;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm < 1) n_sm = 1;
    const int max_blocks = 8 * n_sm;
    const NaView s = view_of(base);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_na_zero<<<grid_for(n_cells, max_blocks), NA_THREADS, 0, st>>>(s, n_cells);
    k_na_sums<<<grid_for(n, max_blocks), NA_THREADS, 0, st>>>(s, cell, v, flags, n, n_cells);
    k_na_dev<<<grid_for(n, max_blocks), NA_THREADS, 0, st>>>(s, cell, v, n, n_cells);
    k_na_cells<<<grid_for(n_cells, max_blocks), NA_THREADS, 0, st>>>(s, n_cells, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(RMPCD_ECUDA, "kernel launch failed (CUDA error %lld)", (long long)e);
    return RMPCD_OK;
}
