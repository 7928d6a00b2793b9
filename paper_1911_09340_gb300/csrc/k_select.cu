// Selection of the k seeds of lowest RSS (Sec. 2.1; top-k as in Sec. 3.1's ten best seeds per side).
//
// Order: ascending RSS, equal RSS by ascending seed index, NaN after every number.  With the index
// as tie-break every key is unique, so round r of a selection is simply "the smallest key greater
// than the key chosen in round r-1".
//
// Pass 1: each block takes a contiguous chunk of the RSS array and runs k rounds of a block argmin
// (per-thread minimum, warp-shuffle reduction, then a shared-memory reduction over the warps),
// writing its k smallest keys to the scratch buffer.  Pass 2: one block runs the same k rounds over
// all blocks' candidates.  Deterministic: no atomics, fixed reduction trees.
#include <float.h>
#include <stdint.h>

#include <mutex>

#include "device.cuh"
#include "internal.h"

namespace comet {

namespace {

constexpr int kSelThreads = 256;
constexpr int kChunk = 2048;
constexpr int64_t kNone = INT64_MAX;

template <typename T>
struct Key {
    T v;
    int64_t i;
};

// a < b in (NaN last, value, index) order; the "none" key (index kNone) is greater than all others.
template <typename T>
__device__ __forceinline__ bool key_less(const Key<T> &a, const Key<T> &b)
{
    if (a.i == kNone || b.i == kNone) return a.i < b.i;
    const bool an = isnan(a.v), bn = isnan(b.v);
    if (an != bn) return bn;
    if (!an && a.v != b.v) return a.v < b.v;
    return a.i < b.i;
}

template <typename T>
__device__ __forceinline__ Key<T> warp_min(Key<T> k)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        Key<T> o;
        o.v = __shfl_xor_sync(0xffffffffu, k.v, off);
        o.i = __shfl_xor_sync(0xffffffffu, k.i, off);
        if (key_less(o, k)) k = o;
    }
    return k;
}

// k rounds of block argmin over the keys produced by get(j) for j in [0, n).  Writes round r's key
// to out_v[r], out_i[r] (thread 0).
template <typename T, class Get>
__device__ void block_topk(int64_t n, int k, Get get, T *out_v, int64_t *out_i)
{
    __shared__ Key<T> red[kSelThreads / 32];
    __shared__ Key<T> last;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) {
        last.v = T(0);
        last.i = -1;      // below every key
    }
    __syncthreads();
    for (int r = 0; r < k; ++r) {
        const Key<T> lk = last;
        Key<T> best{T(0), kNone};
        for (int64_t j = tid; j < n; j += kSelThreads) {
            const Key<T> c = get(j);
            const bool gt = lk.i < 0 || key_less(lk, c);
            if (gt && key_less(c, best)) best = c;
        }
        best = warp_min(best);
        if (lane == 0) red[wid] = best;
        __syncthreads();
        if (wid == 0) {
            Key<T> b = lane < kSelThreads / 32 ? red[lane] : Key<T>{T(0), kNone};
            b = warp_min(b);
            if (lane == 0) {
                out_v[r] = b.v;
                out_i[r] = b.i;
                last = b;
            }
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(kSelThreads) select_pass1(const T *__restrict__ rss, int64_t S,
                                                            int k, T *pv, int64_t *pi)
{
    const int64_t b0 = (int64_t)blockIdx.x * kChunk;
    const int64_t n = min((int64_t)kChunk, S - b0);
    block_topk<T>(n, k, [&](int64_t j) { return Key<T>{rss[b0 + j], b0 + j}; },
                  pv + (int64_t)blockIdx.x * k, pi + (int64_t)blockIdx.x * k);
}

template <typename T>
__global__ void __launch_bounds__(kSelThreads) select_pass2(const T *__restrict__ pv,
                                                            const int64_t *__restrict__ pi,
                                                            int64_t n, int k, int64_t *idx_out,
                                                            T *rss_out)
{
    __shared__ T ov[64];
    __shared__ int64_t oi[64];
    block_topk<T>(n, k, [&](int64_t j) { return Key<T>{pv[j], pi[j]}; }, ov, oi);
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
        idx_out[r] = oi[r];
        if (rss_out) rss_out[r] = ov[r];
    }
}

// A batch: pass 1 block b serves the chunk batch_find gives inside its event; pass 2 block e serves
// event e.  Each event's partial results live at its SelArgs.scratch (ids first, then values).
template <typename T>
__global__ void __launch_bounds__(kSelThreads) select_pass1_batch(BatchLaunch L)
{
    int e;
    int64_t lb;
    if (!batch_find(L.sel_start, L.B, blockIdx.x, e, lb)) return;
    const SelArgs a = L.ev[e].sel;
    int64_t *pi = (int64_t *)a.scratch;
    T *pv = (T *)(pi + (int64_t)a.n_blocks * a.k);
    const T *__restrict__ rss = (const T *)a.rss;
    const int64_t b0 = lb * kChunk;
    const int64_t n = min((int64_t)kChunk, a.S - b0);
    block_topk<T>(n, a.k, [&](int64_t j) { return Key<T>{rss[b0 + j], b0 + j}; }, pv + lb * a.k,
                  pi + lb * a.k);
}

template <typename T>
__global__ void __launch_bounds__(kSelThreads) select_pass2_batch(BatchLaunch L)
{
    if ((int)blockIdx.x >= L.B) return;
    const SelArgs a = L.ev[blockIdx.x].sel;
    if (a.S <= 0) return;
    const int64_t *pi = (const int64_t *)a.scratch;
    const T *pv = (const T *)(pi + (int64_t)a.n_blocks * a.k);
    __shared__ T ov[64];
    __shared__ int64_t oi[64];
    block_topk<T>((int64_t)a.n_blocks * a.k, a.k, [&](int64_t j) { return Key<T>{pv[j], pi[j]}; }, ov, oi);
    for (int r = threadIdx.x; r < a.k; r += blockDim.x) {
        a.idx_out[r] = oi[r];
        if (a.rss_out) ((T *)a.rss_out)[r] = ov[r];
    }
}

} // namespace

cudaError_t launch_select_batch(comet_dtype dt, const BatchLaunch &L, cudaStream_t st)
{
    if (L.B == 0) return cudaSuccess;
    if (dt == COMET_F32) {
        if (L.sel_blocks) select_pass1_batch<float><<<L.sel_blocks, kSelThreads, 0, st>>>(L);
        select_pass2_batch<float><<<(unsigned)L.B, kSelThreads, 0, st>>>(L);
    } else {
        if (L.sel_blocks) select_pass1_batch<double><<<L.sel_blocks, kSelThreads, 0, st>>>(L);
        select_pass2_batch<double><<<(unsigned)L.B, kSelThreads, 0, st>>>(L);
    }
    return cudaGetLastError();
}

int select_chunk() { return kChunk; }

size_t select_scratch_bytes(comet_dtype dt, int64_t S, int k, int *n_blocks)
{
    const int64_t nb = (S + kChunk - 1) / kChunk;
    *n_blocks = (int)nb;
    const size_t es = dt == COMET_F32 ? sizeof(float) : sizeof(double);
    return (size_t)nb * k * (es + sizeof(int64_t)) + 64;
}

template <typename T>
static void sel_launch(const SelArgs &a, cudaStream_t st)
{
    const int nb = a.n_blocks;
    int64_t *pi = (int64_t *)a.scratch;
    T *pv = (T *)(pi + (int64_t)nb * a.k);
    select_pass1<T><<<nb, kSelThreads, 0, st>>>((const T *)a.rss, a.S, a.k, pv, pi);
    select_pass2<T><<<1, kSelThreads, 0, st>>>(pv, pi, (int64_t)nb * a.k, a.k, a.idx_out,
                                              (T *)a.rss_out);
}

// Scratch of comet_scan_select_noalloc: one file-scope device array per device that loads the
// library, held until the process exits.  In host code `g_select_scratch` is only a host-side
// stand-in for the symbol, never a device address: the device address is looked up once per device
// with cudaGetSymbolAddress, with that device current, and cached here.
static __device__ __align__(256) unsigned char g_select_scratch[kStaticSelectScratchBytes];

cudaError_t static_select_scratch(void **ptr)
{
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static void *addr[kMaxDevices] = {};
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_select_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = p;
    }
    *ptr = addr[dev];
    return cudaSuccess;
}

cudaError_t kernel_binary_version(int *version)
{
    cudaFuncAttributes fa;
    const cudaError_t e = cudaFuncGetAttributes(&fa, select_pass1<float>);
    if (e == cudaSuccess) *version = fa.binaryVersion;
    return e;
}

cudaError_t launch_select(comet_dtype dt, const SelArgs &a, cudaStream_t st)
{
    if (dt == COMET_F32)
        sel_launch<float>(a, st);
    else
        sel_launch<double>(a, st);
    return cudaGetLastError();
}

} // namespace comet
