// Quality: the F1-score of a detected cover against a reference cover
// (Methods, Evaluation Criteria, F1-Score for Overlapping Communities): the
// mean over detected communities C' of max over reference communities C of
// F1(C', C) = 2 (p r) / (p + r), p = |C & C'| / |C'|, r = |C & C'| / |C|,
// 0 when they share no node.  Per detected community one block counts
// |C & C'| for every reference community its members belong to, in a shared
// hash table (several passes over hash parts when there are more candidates
// than the table holds); the mean is an exact sum.
#include <vector>

#include "lf_internal.cuh"

namespace lf {
namespace {

constexpr int F1_THREADS = 256;
constexpr uint32_t F1_SLOTS = 4096;

// reference memberships as (node << 32 | community)
__global__ void k_ref_keys(const int64_t *off, const int32_t *mem, int64_t kb, int64_t eb,
                           unsigned long long *keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < eb; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = kb - 1;   // community of entry i: last c with off[c] <= i
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (off[mid] <= i) lo = mid; else hi = mid - 1;
        }
        keys[i] = ((unsigned long long)(uint32_t)mem[i] << 32) | (unsigned long long)lo;
    }
}

__device__ __forceinline__ int64_t first_key(const unsigned long long *keys, int64_t eb, uint32_t node) {
    const unsigned long long k = (unsigned long long)node << 32;
    int64_t lo = 0, hi = eb;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < k) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ double f1_pair(int64_t k, int64_t a, int64_t b) {
    if (k == 0) return 0.0;
    const double p = __ddiv_rn((double)k, (double)a), r = __ddiv_rn((double)k, (double)b);
    return __dmul_rn(2.0, __ddiv_rn(__dmul_rn(p, r), __dadd_rn(p, r)));
}

// (score descending, reference index ascending); c < 0 = none
__device__ __forceinline__ bool f1_better(double f1, int32_t c1, double f2, int32_t c2) {
    if (c1 < 0) return false;
    if (c2 < 0) return true;
    return f1 > f2 || (f1 == f2 && c1 < c2);
}

__global__ void __launch_bounds__(F1_THREADS) k_cover_f1(const int64_t *off_a, const int32_t *mem_a, int64_t ka,
                                                         const int64_t *off_b, const unsigned long long *keys,
                                                         int64_t eb, unsigned long long *sacc, int32_t *best) {
    __shared__ int32_t hk[F1_SLOTS];
    __shared__ uint32_t hv[F1_SLOTS];
    __shared__ double s_f[F1_THREADS / 32];
    __shared__ int32_t s_c[F1_THREADS / 32];
    __shared__ unsigned long long s_bound;
    __shared__ int s_over;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t c = blockIdx.x; c < ka; c += gridDim.x) {
        const int64_t beg = off_a[c], end = off_a[c + 1], a = end - beg;
        // candidates bound: the members' reference memberships
        if (threadIdx.x == 0) s_bound = 0;
        __syncthreads();
        unsigned long long mine = 0;
        for (int64_t i = beg + threadIdx.x; i < end; i += F1_THREADS) {
            const uint32_t x = (uint32_t)mem_a[i];
            const int64_t lo = first_key(keys, eb, x);
            const int64_t hi = first_key(keys, eb, x + 1u == 0u ? 0xffffffffu : x + 1u);
            mine += (unsigned long long)((x == 0xffffffffu ? eb : hi) - lo);
        }
        atomicAdd(&s_bound, mine);
        __syncthreads();
        const unsigned long long bound = s_bound;
        uint32_t P = bound <= F1_SLOTS / 2 ? 1u : (uint32_t)((bound + F1_SLOTS / 2 - 1) / (F1_SLOTS / 2));
        double bf = 0.0;
        int32_t bc = -1;
        for (;;) {   // a part that overflows the table makes the parts twice as many
        bf = 0.0;
        bc = -1;
        if (threadIdx.x == 0) s_over = 0;
        for (uint32_t part = 0; part < P; ++part) {
            for (uint32_t s = threadIdx.x; s < F1_SLOTS; s += F1_THREADS) {
                hk[s] = -1;
                hv[s] = 0u;
            }
            __syncthreads();
            for (int64_t i = beg + threadIdx.x; i < end; i += F1_THREADS) {
                const uint32_t x = (uint32_t)mem_a[i];
                for (int64_t j = first_key(keys, eb, x); j < eb && (uint32_t)(keys[j] >> 32) == x; ++j) {
                    const int32_t cb = (int32_t)(keys[j] & 0xffffffffull);
                    if (P > 1 && hash32((uint32_t)cb ^ 0x85ebca6bu) % P != part) continue;
                    uint32_t h = hash32((uint32_t)cb) & (F1_SLOTS - 1);
                    bool placed = false;
                    for (uint32_t probe = 0; probe < F1_SLOTS; ++probe) {
                        const int32_t prev = atomicCAS(&hk[h], -1, cb);
                        if (prev == -1 || prev == cb) {
                            atomicAdd(&hv[h], 1u);
                            placed = true;
                            break;
                        }
                        h = (h + 1) & (F1_SLOTS - 1);
                    }
                    if (!placed) s_over = 1;
                }
            }
            __syncthreads();
            for (uint32_t s = threadIdx.x; s < F1_SLOTS; s += F1_THREADS) {
                const int32_t cb = hk[s];
                if (cb < 0) continue;
                const double f = f1_pair(hv[s], a, off_b[cb + 1] - off_b[cb]);
                if (f1_better(f, cb, bf, bc)) {
                    bf = f;
                    bc = cb;
                }
            }
            __syncthreads();
        }
        if (!s_over) break;
        __syncthreads();
        P *= 2;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double f2 = __shfl_down_sync(FULL, bf, o);
            const int32_t c2 = __shfl_down_sync(FULL, bc, o);
            if (f1_better(f2, c2, bf, bc)) {
                bf = f2;
                bc = c2;
            }
        }
        if (lane == 0) {
            s_f[w] = bf;
            s_c[w] = bc;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 1; k < F1_THREADS / 32; ++k)
                if (f1_better(s_f[k], s_c[k], bf, bc)) {
                    bf = s_f[k];
                    bc = s_c[k];
                }
            if (best) best[c] = bc;
            sacc_add(sacc, bc >= 0 ? bf : 0.0);
        }
        __syncthreads();
    }
}

__global__ void k_f1_final(unsigned long long *sacc, int64_t ka, double *out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const double s = sacc_round_and_clear(sacc);
    *out = ka > 0 ? __ddiv_rn(s, (double)ka) : 0.0;
}

}  // namespace
}  // namespace lf

extern "C" lf_status lf_cover_f1(const int64_t *det_offsets, const int32_t *det_members, int64_t num_det,
                                 const int64_t *ref_offsets, const int32_t *ref_members, int64_t num_ref,
                                 double *f1, int32_t *best, void *stream) {
    using namespace lf;
    if (!f1 || num_det < 0 || num_ref < 0 || (num_det > 0 && !det_offsets) || (num_ref > 0 && !ref_offsets)) {
        set_error(LF_ERR_INVALID, "invalid argument");
        return LF_ERR_INVALID;
    }
    *f1 = 0.0;
    if (num_det == 0) return LF_OK;
    lf_graph tmp;   // allocation and launch bookkeeping for the call
    tmp.stream = static_cast<cudaStream_t>(stream);
    bool own = false;
    std::vector<void *> bufs;
    lf_status rc = LF_OK;
    try {
        if (!tmp.stream) {
            LF_CUDA(cudaStreamCreateWithFlags(&tmp.stream, cudaStreamNonBlocking));
            own = true;
        }
        cudaStream_t st = tmp.stream;
        const int64_t ea = det_offsets[num_det], eb = num_ref > 0 ? ref_offsets[num_ref] : 0;
        if (det_offsets[0] != 0 || (num_ref > 0 && ref_offsets[0] != 0)) fail(LF_ERR_INVALID, "offsets must start at 0");
        if ((ea > 0 && !det_members) || (eb > 0 && !ref_members)) fail(LF_ERR_INVALID, "members is NULL");
        for (int64_t c = 0; c < num_det; ++c)
            if (det_offsets[c + 1] <= det_offsets[c]) fail(LF_ERR_INVALID, "detected community %lld is empty", (long long)c);
        for (int64_t c = 0; c < num_ref; ++c)
            if (ref_offsets[c + 1] <= ref_offsets[c]) fail(LF_ERR_INVALID, "reference community %lld is empty", (long long)c);
        uint32_t max_id = 0;
        for (int64_t i = 0; i < ea; ++i) {
            if (det_members[i] < 0) fail(LF_ERR_INVALID, "negative node id");
            max_id = std::max(max_id, (uint32_t)det_members[i]);
        }
        for (int64_t i = 0; i < eb; ++i) {
            if (ref_members[i] < 0) fail(LF_ERR_INVALID, "negative node id");
            max_id = std::max(max_id, (uint32_t)ref_members[i]);
        }
        auto alloc = [&](size_t bytes) {
            void *d = dalloc(&tmp, bytes > 0 ? bytes : 8);
            bufs.push_back(d);
            return d;
        };
        auto up = [&](const void *h, size_t bytes) {   // a device copy of host data
            void *d = alloc(bytes);
            if (bytes) LF_CUDA(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, st));
            return d;
        };
        auto *oa = static_cast<int64_t *>(up(det_offsets, (size_t)(num_det + 1) * 8));
        auto *ma = static_cast<int32_t *>(up(det_members, (size_t)ea * 4));
        auto *ob = static_cast<int64_t *>(num_ref > 0 ? up(ref_offsets, (size_t)(num_ref + 1) * 8) : alloc(8));
        auto *mb = static_cast<int32_t *>(up(ref_members, (size_t)eb * 4));
        auto *keys = static_cast<unsigned long long *>(alloc((size_t)eb * 8));
        auto *sacc = static_cast<unsigned long long *>(alloc(SACC_CHUNKS * 8));
        auto *bst = static_cast<int32_t *>(alloc((size_t)num_det * 4));
        auto *res = static_cast<double *>(alloc(8));
        LF_CUDA(cudaMemsetAsync(sacc, 0, SACC_CHUNKS * 8, st));
        if (eb > 0) {
            k_ref_keys<<<grid_for(eb, 256, 1 << 16), 256, 0, st>>>(ob, mb, num_ref, eb, keys);
            LF_LAUNCHED();
            std::vector<int> sh;
            for (int s = 0; s < bits_for((unsigned long long)(num_ref - 1)); s += 8) sh.push_back(s);
            for (int s = 0; s < bits_for((unsigned long long)max_id); s += 8) sh.push_back(32 + s);
            radix_sort(&tmp, keys, nullptr, eb, sh);
        }
        k_cover_f1<<<grid_for(num_det, 1, 152 * 8), F1_THREADS, 0, st>>>(oa, ma, num_det, ob, keys, eb, sacc, bst);
        LF_LAUNCHED();
        k_f1_final<<<1, 32, 0, st>>>(sacc, num_det, res);
        LF_LAUNCHED();
        LF_CUDA(cudaMemcpyAsync(f1, res, 8, cudaMemcpyDeviceToHost, st));
        if (best) LF_CUDA(cudaMemcpyAsync(best, bst, (size_t)num_det * 4, cudaMemcpyDeviceToHost, st));
        LF_CUDA(cudaStreamSynchronize(st));
    } catch (const Error &e) {
        rc = e.status;
    } catch (...) {
        set_error(LF_ERR_CUDA, "unexpected internal error");
        rc = LF_ERR_CUDA;
    }
    for (void *p : bufs) dfree(&tmp, p);
    if (tmp.stream) cudaStreamSynchronize(tmp.stream);
    if (own) cudaStreamDestroy(tmp.stream);
    return rc;
}
