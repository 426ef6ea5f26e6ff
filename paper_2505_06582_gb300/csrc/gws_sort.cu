// gws_sort.cu -- stable LSD radix sort (8-bit digits) of (key, u32 value) pairs.
//
// Used for the depth sort (front = smallest mu_z first, ties keep input order, as
// Algorithm S2 orders the Gaussians front to back), for ordering each wavelength's
// records by spectral footprint radius, and for ordering the splat work items.
// Each pass: per-block digit histogram -> one-block exclusive scan (digit-major) ->
// stable scatter (in-block ranks from warp match_any, warps in order, rounds in order).
#include "gws_host.h"

namespace gws {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const K *__restrict__ keys, long long n, int shift,
                                                            unsigned *__restrict__ hist, int nblocks) {
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kSortTile;
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        long long idx = base + k * kSortThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[(unsigned)((keys[idx] >> shift) & 255u)], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of `total` u32 in place, one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_sort_scan(unsigned *__restrict__ data, long long total) {
    __shared__ unsigned warp_tot[32];
    __shared__ unsigned carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (long long base = 0; base < total; base += 4096) {
        unsigned v[4];
        const long long i0 = base + (long long)tid * 4;
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = (i0 + k < total) ? data[i0 + k] : 0u;
        unsigned s = v[0] + v[1] + v[2] + v[3];
        unsigned inc = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) warp_tot[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            unsigned w = warp_tot[lane];
            unsigned wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            warp_tot[lane] = wi - w;  // exclusive warp offsets
        }
        __syncthreads();
        unsigned run = carry + warp_tot[warp] + inc - s;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (i0 + k < total) data[i0 + k] = run;
            run += v[k];
        }
        __syncthreads();
        if (tid == 1023) carry = run;
        __syncthreads();
    }
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads)
    k_sort_scatter(const K *__restrict__ keys_in, const unsigned *__restrict__ vals_in, K *__restrict__ keys_out,
                   unsigned *__restrict__ vals_out, long long n, int shift, const unsigned *__restrict__ offs,
                   int nblocks, int *status) {
    __shared__ unsigned s_off[256];
    __shared__ unsigned s_wc[kSortThreads / 32][257];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_off[tid] = offs[(size_t)tid * nblocks + blockIdx.x];
    for (int i = tid; i < (kSortThreads / 32) * 257; i += kSortThreads) (&s_wc[0][0])[i] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    const long long base = (long long)blockIdx.x * kSortTile;
    for (int k = 0; k < kSortItems; ++k) {
        const long long idx = base + k * kSortThreads + tid;
        const bool valid = idx < n;
        K key = valid ? keys_in[idx] : K(0);
        unsigned val = valid ? vals_in[idx] : 0u;
        unsigned d = valid ? (unsigned)((key >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned rank = __popc(peers & lt);
        if (lane == __ffs(peers) - 1) s_wc[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            unsigned pos = s_off[d] + rank;
            for (int w = 0; w < warp; ++w) pos += s_wc[w][d];
            if (in_bounds((long long)pos < n, status)) {
                keys_out[pos] = key;
                vals_out[pos] = val;
            }
        }
        __syncthreads();
        {
            unsigned t = 0;
#pragma unroll
            for (int w = 0; w < kSortThreads / 32; ++w) {
                t += s_wc[w][tid];
                s_wc[w][tid] = 0;
            }
            s_off[tid] += t;
            if (tid < kSortThreads / 32) s_wc[tid][256] = 0;
        }
        __syncthreads();
    }
}

size_t sort_hist_words(long long n) {
    long long nb = (n + kSortTile - 1) / kSortTile;
    if (nb < 1) nb = 1;
    return (size_t)256 * (size_t)nb;
}

template <typename K>
cudaError_t radix_sort(K *&keys, K *&keys_alt, unsigned *&vals, unsigned *&vals_alt, long long n, int begin_bit,
                       int end_bit, unsigned *hist, cudaStream_t s, int *status) {
    if (n <= 1) return cudaSuccess;
    const int nb = (int)((n + kSortTile - 1) / kSortTile);
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
        k_sort_hist<K><<<nb, kSortThreads, 0, s>>>(keys, n, shift, hist, nb);
        k_sort_scan<<<1, 1024, 0, s>>>(hist, (long long)256 * nb);
        k_sort_scatter<K><<<nb, kSortThreads, 0, s>>>(keys, vals, keys_alt, vals_alt, n, shift, hist, nb, status);
        count_launches(3);
        K *tk = keys;
        keys = keys_alt;
        keys_alt = tk;
        unsigned *tv = vals;
        vals = vals_alt;
        vals_alt = tv;
    }
    return cudaGetLastError();
}

template cudaError_t radix_sort<unsigned>(unsigned *&, unsigned *&, unsigned *&, unsigned *&, long long, int, int,
                                          unsigned *, cudaStream_t, int *);
template cudaError_t radix_sort<unsigned long long>(unsigned long long *&, unsigned long long *&, unsigned *&,
                                                    unsigned *&, long long, int, int, unsigned *, cudaStream_t, int *);

}  // namespace gws
