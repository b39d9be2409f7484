// scan.cu -- device-wide exclusive scan and stable LSD radix sort (build-time primitives).
//
// The canonical reduction of Sec. 2.3 sorts the (X, Z) keys with a radix sort;
// this is that sort, written for the GPU: 8-bit digits, one pass per digit,
// each pass a tile histogram, a scan of the digit-major histogram and a stable
// scatter in which every tile ranks its elements warp by warp in index order.
#include "ps_internal.cuh"

namespace ps {
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of the per-thread values of one block.
__device__ void block_excl_scan(int64_t v, int64_t *exclusive) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = warp_incl_scan(v);
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = (lane < kScanThreads / 32) ? warp_tot[lane] : 0;
        int64_t wi = warp_incl_scan(w);
        if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;
    }
    __syncthreads();
    *exclusive = warp_tot[warp] + incl - v;
}

__global__ void k_tile_sums(const int64_t *in, int64_t n, int64_t *sums) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    __shared__ int64_t red[kScanThreads];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kScanThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = red[0];
}

__global__ void k_tile_scan(const int64_t *in, int64_t n, const int64_t *tile_off, int64_t *out) {
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        s += v[i];
    }
    int64_t ex;
    block_excl_scan(s, &ex);
    int64_t run = ex + (tile_off ? tile_off[blockIdx.x] : 0);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

// ---------------------------------------------------------------------------
// radix sort
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;
constexpr int kSortTile = kSortThreads * kSortRounds;
constexpr int kSortWarps = kSortThreads / 32;

__device__ __forceinline__ int digit_of(uint64_t hi, uint64_t lo, int bit) {
    return bit < 64 ? (int)((lo >> bit) & 0xffu) : (int)((hi >> (bit - 64)) & 0xffu);
}

__global__ void k_radix_hist(const uint64_t *hi, const uint64_t *lo, int64_t n, int bit,
                             int64_t ntiles, int64_t *hist) {
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; ++r) {
        int64_t i = base + r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[digit_of(hi[i], lo[i], bit)], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_radix_scatter(const uint64_t *hi, const uint64_t *lo, const int64_t *perm,
                                int64_t n, int bit, int64_t ntiles, const int64_t *offs,
                                uint64_t *ohi, uint64_t *olo, int64_t *operm) {
    __shared__ int wcount[kSortWarps][256];
    __shared__ int64_t base_cnt[256];
    __shared__ int round_tot[256];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int w = 0; w < kSortWarps; ++w) wcount[w][t] = 0;
    base_cnt[t] = offs[(int64_t)t * ntiles + blockIdx.x];
    __syncthreads();
    const unsigned lt_mask = (1u << lane) - 1u;
    int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; ++r) {
        int64_t i = tile0 + r * kSortThreads + t;
        bool valid = i < n;
        uint64_t h = 0, l = 0;
        int64_t p = 0;
        int d = 256 + lane;  // unique sentinel per lane for invalid elements
        if (valid) {
            h = hi[i];
            l = lo[i];
            p = perm[i];
            d = digit_of(h, l, bit);
        }
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank_in_warp = __popc(peers & lt_mask);
        if (valid && rank_in_warp == 0) wcount[warp][d] = __popc(peers);
        __syncthreads();
        {
            int pre = 0;
            for (int w = 0; w < kSortWarps; ++w) {
                int c = wcount[w][t];
                wcount[w][t] = pre;
                pre += c;
            }
            round_tot[t] = pre;
        }
        __syncthreads();
        if (valid) {
            int64_t pos = base_cnt[d] + wcount[warp][d] + rank_in_warp;
            ohi[pos] = h;
            olo[pos] = l;
            operm[pos] = p;
        }
        __syncthreads();
        base_cnt[t] += round_tot[t];
        for (int w = 0; w < kSortWarps; ++w) wcount[w][t] = 0;
        __syncthreads();
    }
}

__global__ void k_iota(int64_t *p, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = i;
}

}  // namespace

void exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, const Allocator &al,
                        cudaStream_t st) {
    if (n <= 0) return;
    int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles == 1) {
        k_tile_scan<<<1, kScanThreads, 0, st>>>(in, n, nullptr, out);
        PS_LAUNCH_CHECK();
        return;
    }
    DevBuf<int64_t> sums(al, ntiles), offs(al, ntiles);
    k_tile_sums<<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, n, sums.p);
    PS_LAUNCH_CHECK();
    exclusive_scan_i64(sums.p, offs.p, ntiles, al, st);
    k_tile_scan<<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, n, offs.p, out);
    PS_LAUNCH_CHECK();
    PS_CUDA(cudaStreamSynchronize(st));  // temporaries are released on return
}

void radix_sort_keys(uint64_t *hi, uint64_t *lo, int64_t *perm, int64_t n, int hi_bits, int lo_bits,
                     const Allocator &al, cudaStream_t st) {
    if (n <= 0) return;
    k_iota<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(perm, n);
    PS_LAUNCH_CHECK();
    std::vector<int> passes;
    for (int b = 0; b < lo_bits; b += 8) passes.push_back(b);
    for (int b = 0; b < hi_bits; b += 8) passes.push_back(64 + b);
    if (passes.empty() || n == 1) return;
    int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    DevBuf<uint64_t> hi2(al, n), lo2(al, n);
    DevBuf<int64_t> perm2(al, n), hist(al, 256 * ntiles), offs(al, 256 * ntiles);
    uint64_t *ch = hi, *cl = lo, *nh = hi2.p, *nl = lo2.p;
    int64_t *cp = perm, *np = perm2.p;
    for (int bit : passes) {
        k_radix_hist<<<(unsigned)ntiles, kSortThreads, 0, st>>>(ch, cl, n, bit, ntiles, hist.p);
        PS_LAUNCH_CHECK();
        exclusive_scan_i64(hist.p, offs.p, 256 * ntiles, al, st);
        k_radix_scatter<<<(unsigned)ntiles, kSortThreads, 0, st>>>(ch, cl, cp, n, bit, ntiles, offs.p,
                                                                     nh, nl, np);
        PS_LAUNCH_CHECK();
        std::swap(ch, nh);
        std::swap(cl, nl);
        std::swap(cp, np);
    }
    if (ch != hi) {
        PS_CUDA(cudaMemcpyAsync(hi, ch, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
        PS_CUDA(cudaMemcpyAsync(lo, cl, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
        PS_CUDA(cudaMemcpyAsync(perm, cp, n * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    }
    PS_CUDA(cudaStreamSynchronize(st));
}

}  // namespace ps
