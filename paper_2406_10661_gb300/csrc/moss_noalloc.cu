// moss_lane_offsets_noalloc: the lane-offset scan of the step (the work of
// k_lanescan) for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits — inside a
// framework whose caching allocator owns the device memory, in a process with
// a fixed memory reservation, or in a pipeline that must not allocate between
// its own set-up and teardown.  Such a caller owns the per-lane input and
// output arrays; the only extra memory this call needs, the look-back words
// of the single-pass scan, lives in a file-scope static device array that
// every GPU loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "moss.h"
#include "moss_device.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_ITEMS = 4;
constexpr int NA_TILE = NA_THREADS * NA_ITEMS;
constexpr int NA_MAX_TILES = MOSS_NOALLOC_MAX_LANES / NA_TILE;
constexpr int NA_MAX_DEVICES = 64;

struct NoallocScratch {
    unsigned long long tile[NA_MAX_TILES];  // look-back words: flag:2 | leavers:31 | sizes:31
    int ticket;                             // dynamic tile counter
    int err;                                // a bounded wait gave up, or a lane's new size was negative
    int pad[62];
};

// 32 KiB + 256 B of scratch per device, shared by every call
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

std::mutex g_mu;
NoallocScratch* g_ptr[NA_MAX_DEVICES] = {};
int g_sms[NA_MAX_DEVICES] = {};

__global__ void k_noalloc_clear(NoallocScratch* sc, int ntiles) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ntiles; k += gridDim.x * blockDim.x)
        sc->tile[k] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->ticket = 0;
        sc->err = 0;
    }
}

// a wait that gave up marks the whole result invalid (documented sentinel)
__global__ void k_noalloc_finish(const NoallocScratch* sc, int32_t* off_next, int n) {
    if (sc->err) off_next[n] = -1;
}

// newsize(l) = off_cur[l+1] - off_cur[l] - leave[l] + enter[l];
// off_next = exclusive scan of newsize (n+1 entries), lbefore = exclusive scan of leave.
__global__ void __launch_bounds__(NA_THREADS) k_noalloc_lanescan(NoallocScratch* sc, int n, int ntiles,
                                                                 const int32_t* off_cur,
                                                                 const int32_t* leave,
                                                                 const int32_t* enter,
                                                                 int32_t* off_next, int32_t* lbefore) {
    __shared__ int s_tile;
    __shared__ long long s_sum[NA_THREADS];
    __shared__ unsigned long long s_prefix;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&sc->ticket, 1);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= ntiles) return;
        const int base = tile * NA_TILE + threadIdx.x * NA_ITEMS;
        int ns[NA_ITEMS], lv[NA_ITEMS];
        long long tn = 0, tl = 0;
#pragma unroll
        for (int k = 0; k < NA_ITEMS; ++k) {
            const int l = base + k;
            if (l < n) {
                lv[k] = leave[l];
                ns[k] = off_cur[l + 1] - off_cur[l] - lv[k] + enter[l];
                if (ns[k] < 0) {  // violated precondition: reported, and kept out of the packed sums
                    atomicOr(&sc->err, 2);
                    ns[k] = 0;
                }
            } else {
                ns[k] = 0; lv[k] = 0;
            }
            tn += ns[k]; tl += lv[k];
        }
        const long long packed = (tl << 31) | tn;
        s_sum[threadIdx.x] = packed;
        __syncthreads();
        for (int o = 1; o < NA_THREADS; o <<= 1) {
            const long long x = threadIdx.x >= o ? s_sum[threadIdx.x - o] : 0;
            __syncthreads();
            s_sum[threadIdx.x] += x;
            __syncthreads();
        }
        const long long incl = s_sum[threadIdx.x];
        const long long total = s_sum[NA_THREADS - 1];
        if (threadIdx.x == 0) {
            unsigned long long prefix = 0;
            if (tile == 0) {
                moss::store_release(&sc->tile[0], (2ull << 62) | (unsigned long long)total);
            } else {
                moss::store_release(&sc->tile[tile], (1ull << 62) | (unsigned long long)total);
                int p = tile - 1;
                long long spins = 0;
                while (p >= 0) {
                    const unsigned long long w = moss::load_acquire(&sc->tile[p]);
                    const unsigned long long f = w >> 62;
                    if (f == 0) {
                        if (++spins > moss::SPIN_LIMIT) { atomicOr(&sc->err, 1); break; }
                        if (spins > 64) __nanosleep(100);
                        continue;
                    }
                    prefix += w & ((1ull << 62) - 1);
                    if (f == 2) break;
                    --p;
                }
                moss::store_release(&sc->tile[tile], (2ull << 62) | (prefix + (unsigned long long)total));
            }
            s_prefix = prefix;
        }
        __syncthreads();
        long long excl = (long long)s_prefix + incl - packed;
        long long en = excl & ((1ll << 31) - 1), el = excl >> 31;
#pragma unroll
        for (int k = 0; k < NA_ITEMS; ++k) {
            const int l = base + k;
            if (l < n) {
                off_next[l] = (int)en;
                lbefore[l] = (int)el;
            }
            en += ns[k]; el += lv[k];
        }
        if (tile == ntiles - 1 && threadIdx.x == NA_THREADS - 1) off_next[n] = (int)en;
        __syncthreads();
    }
}

// once per device, with that device current: the device address of the
// static scratch (a host-side name of a __device__ variable is not a device
// address) and the SM count used to size the grid
int setup_device(int dev, NoallocScratch** out, int* sms) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return MOSS_ECUDA;
        }
        int s = 0;
        if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return MOSS_ECUDA;
        }
        g_ptr[dev] = (NoallocScratch*)p;
        g_sms[dev] = s;
    }
    *out = g_ptr[dev];
    *sms = g_sms[dev];
    return MOSS_OK;
}

}  // namespace

extern "C" int moss_lane_offsets_noalloc(int32_t n_lanes, const int32_t* d_off_cur,
                                         const int32_t* d_leave, const int32_t* d_enter,
                                         int32_t* d_off_next, int32_t* d_lbefore, void* cuda_stream) {
    if (n_lanes < 0 || n_lanes > MOSS_NOALLOC_MAX_LANES) return MOSS_EINVAL;
    if (!d_off_cur || !d_off_next || (n_lanes > 0 && (!d_leave || !d_enter || !d_lbefore)))
        return MOSS_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        cudaGetLastError();
        return MOSS_ECUDA;
    }
    NoallocScratch* sc = nullptr;
    int sms = 1;
    const int rc = setup_device(dev, &sc, &sms);
    if (rc != MOSS_OK) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int ntiles = (n_lanes + NA_TILE - 1) / NA_TILE;
    if (ntiles == 0) {
        // no lanes: the offset array is the single entry 0
        if (cudaMemsetAsync(d_off_next, 0, sizeof(int32_t), s) != cudaSuccess) {
            cudaGetLastError();
            return MOSS_ECUDA;
        }
        return MOSS_OK;
    }
    k_noalloc_clear<<<(ntiles + 255) / 256, 256, 0, s>>>(sc, ntiles);
    const int grid = ntiles < sms * 4 ? ntiles : sms * 4;
    k_noalloc_lanescan<<<grid, NA_THREADS, 0, s>>>(sc, n_lanes, ntiles, d_off_cur, d_leave, d_enter,
                                                   d_off_next, d_lbefore);
    k_noalloc_finish<<<1, 1, 0, s>>>(sc, d_off_next, n_lanes);
    if (cudaGetLastError() != cudaSuccess) return MOSS_ECUDA;
    return MOSS_OK;
}
