// Device primitives: exclusive prefix sum and a stable LSD radix sort of
// 64-bit keys with optional 32-bit payloads.  Hand-written for sm_103a; used
// by the CSR build, the node order and the community output.
#include "lf_internal.cuh"

namespace lf {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ T block_exclusive_scan(T v, T *warp_sums, T &block_total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        T s = lane < SCAN_THREADS / 32 ? warp_sums[lane] : T(0);
#pragma unroll
        for (int o = 1; o < SCAN_THREADS / 32; o <<= 1) {
            T y = __shfl_up_sync(FULL, s, o);
            if (lane >= o) s += y;
        }
        if (lane < SCAN_THREADS / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    T prefix = w > 0 ? warp_sums[w - 1] : T(0);
    block_total = warp_sums[SCAN_THREADS / 32 - 1];
    __syncthreads();
    return prefix + x - v;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const T *in, int64_t count, T *sums) {
    __shared__ T ws[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < count) s += in[base + i];
    T tot;
    block_exclusive_scan<T>(s, ws, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const T *in, T *out, int64_t count,
                                                            const T *block_offsets, T *d_total) {
    __shared__ T ws[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T vals[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        vals[i] = base + i < count ? in[base + i] : T(0);
        s += vals[i];
    }
    T tot;
    T run = block_exclusive_scan<T>(s, ws, tot);
    T boff = block_offsets ? block_offsets[blockIdx.x] : T(0);
    run += boff;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < count) out[base + i] = run;
        run += vals[i];
    }
    if (d_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *d_total = boff + tot;
}

}  // namespace

template <typename T>
void scan_exclusive(lf_graph *g, const T *in, T *out, int64_t count, T *d_total) {
    if (count <= 0) {
        if (d_total) LF_CUDA(cudaMemsetAsync(d_total, 0, sizeof(T), g->stream));
        return;
    }
    int64_t nb = (count + SCAN_TILE - 1) / SCAN_TILE;
    if (nb > 0x7fffffff) fail(LF_ERR_CAPACITY, "scan of %lld elements", (long long)count);
    if (nb == 1) {
        k_scan_down<T><<<1, SCAN_THREADS, 0, g->stream>>>(in, out, count, nullptr, d_total);
        LF_LAUNCHED();
        g->launches += 1;
        return;
    }
    T *sums = dalloc_n<T>(g, nb);
    k_scan_reduce<T><<<(unsigned)nb, SCAN_THREADS, 0, g->stream>>>(in, count, sums);
    LF_LAUNCHED();
    scan_exclusive<T>(g, sums, sums, nb, nullptr);
    k_scan_down<T><<<(unsigned)nb, SCAN_THREADS, 0, g->stream>>>(in, out, count, sums, d_total);
    LF_LAUNCHED();
    g->launches += 2;
    dfree(g, sums);
}

template void scan_exclusive<int32_t>(lf_graph *, const int32_t *, int32_t *, int64_t, int32_t *);
template void scan_exclusive<uint32_t>(lf_graph *, const uint32_t *, uint32_t *, int64_t, uint32_t *);
template void scan_exclusive<int64_t>(lf_graph *, const int64_t *, int64_t *, int64_t, int64_t *);
template void scan_exclusive<unsigned long long>(lf_graph *, const unsigned long long *,
                                                 unsigned long long *, int64_t, unsigned long long *);

// ---------------------------------------------------------------------------
// LSD radix sort, 8-bit digits.  Per pass: block digit histograms (digit-major
// so that one exclusive scan gives every block its output offset per digit),
// then a stable scatter.  Each warp owns a contiguous sub-tile; inside it,
// equal digits in a 32-item chunk are grouped with __match_any_sync, so the
// rank of an item is (warp's running count for the digit) + (lanes below it
// with the same digit).  Warps, chunks and lanes are visited in input order,
// which keeps the sort stable.
// ---------------------------------------------------------------------------
namespace {

constexpr int RS_WARPS = 8;
constexpr int RS_ITEMS = 8;
constexpr int RS_THREADS = RS_WARPS * 32;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const unsigned long long *keys, int64_t count,
                                                        int shift, uint32_t *counts, int nb) {
    __shared__ uint32_t h[256];
    for (int i = threadIdx.x; i < 256; i += RS_THREADS) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int k = threadIdx.x; k < RS_TILE; k += RS_THREADS) {
        int64_t idx = base + k;
        if (idx < count) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += RS_THREADS) counts[(int64_t)i * nb + blockIdx.x] = h[i];
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const unsigned long long *kin, const uint32_t *vin,
                                                           unsigned long long *kout, uint32_t *vout,
                                                           int64_t count, int shift, const uint32_t *offs,
                                                           int nb) {
    __shared__ uint32_t wh[RS_WARPS][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) wh[i >> 8][i & 255] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * (32 * RS_ITEMS);
    unsigned long long k[RS_ITEMS];
    uint32_t v[RS_ITEMS];
    int dg[RS_ITEMS];
#pragma unroll
    for (int c = 0; c < RS_ITEMS; ++c) {
        int64_t idx = base + c * 32 + lane;
        bool valid = idx < count;
        k[c] = valid ? kin[idx] : 0ull;
        v[c] = (valid && vin) ? vin[idx] : 0u;
        dg[c] = valid ? (int)((k[c] >> shift) & 255u) : 256 + lane;
        unsigned mask = __match_any_sync(FULL, dg[c]);
        if (valid && lane == __ffs(mask) - 1) wh[w][dg[c]] += __popc(mask);
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += RS_THREADS) {
        uint32_t run = offs[(int64_t)d * nb + blockIdx.x];
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ++ww) {
            uint32_t t = wh[ww][d];
            wh[ww][d] = run;
            run += t;
        }
    }
    __syncthreads();
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int c = 0; c < RS_ITEMS; ++c) {
        bool valid = dg[c] < 256;
        unsigned mask = __match_any_sync(FULL, dg[c]);
        if (valid) {
            uint32_t dst = wh[w][dg[c]] + __popc(mask & lt);
            kout[dst] = k[c];
            if (vout) vout[dst] = v[c];
        }
        __syncwarp();
        if (valid && lane == __ffs(mask) - 1) wh[w][dg[c]] += __popc(mask);
        __syncwarp();
    }
}

}  // namespace

int bits_for(unsigned long long max_value) {
    int b = 0;
    while (b < 64 && (max_value >> b) != 0ull) ++b;
    return b;
}

void radix_sort(lf_graph *g, unsigned long long *keys, uint32_t *vals, int64_t count,
                const std::vector<int> &shifts) {
    if (count <= 1 || shifts.empty()) return;
    if (count > 0xffffffffll) fail(LF_ERR_CAPACITY, "radix sort of %lld keys", (long long)count);
    const int64_t nb64 = (count + RS_TILE - 1) / RS_TILE;
    const int nb = (int)nb64;
    unsigned long long *k2 = dalloc_n<unsigned long long>(g, count);
    uint32_t *v2 = vals ? dalloc_n<uint32_t>(g, count) : nullptr;
    uint32_t *counts = dalloc_n<uint32_t>(g, (int64_t)256 * nb);
    unsigned long long *ka = keys, *kb = k2;
    uint32_t *va = vals, *vb = v2;
    for (int shift : shifts) {
        k_rs_hist<<<nb, RS_THREADS, 0, g->stream>>>(ka, count, shift, counts, nb);
        LF_LAUNCHED();
        scan_exclusive<uint32_t>(g, counts, counts, (int64_t)256 * nb, nullptr);
        k_rs_scatter<<<nb, RS_THREADS, 0, g->stream>>>(ka, va, kb, vb, count, shift, counts, nb);
        LF_LAUNCHED();
        g->launches += 2;
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        LF_CUDA(cudaMemcpyAsync(keys, ka, (size_t)count * sizeof(unsigned long long),
                                cudaMemcpyDeviceToDevice, g->stream));
        if (vals)
            LF_CUDA(cudaMemcpyAsync(vals, va, (size_t)count * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                                    g->stream));
    }
    dfree(g, counts);
    if (v2) dfree(g, v2);
    dfree(g, k2);
}

}  // namespace lf
