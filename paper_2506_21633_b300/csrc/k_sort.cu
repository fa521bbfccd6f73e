// k_sort.cu -- step a6 of the rasterizer: depth sort per view, emission of
// the (plane, view, tile) instances in depth order, stable radix sort of the
// instances by tile, per-tile ranges (the depth-indexed Gaussian lists of
// Section II-A of SAR-GS).
//
// Everything here is HBM-bound integer work: exclusive scans, 8-bit LSD radix
// passes (per-block digit histograms, one device-wide scan, stable
// block-local ranking staged in shared memory, coalesced scatter).
#include "sdgr_internal.cuh"

namespace sdgr {

// ---------------------------------------------------------------------------
// Block-wide exclusive scan of one value per thread (blockDim.x = 256).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T x, T *total) {
    __shared__ T warp_tot[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        T t = lane < nw ? warp_tot[lane] : T(0);
        T ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < nw) warp_tot[lane] = ti - t;  // exclusive warp offsets
        if (lane == nw - 1) warp_tot[31] = ti;    // block total
    }
    __syncthreads();
    T res = warp_tot[warp] + inc - x;
    if (total) *total = warp_tot[31];
    __syncthreads();
    return res;
}

// ---------------------------------------------------------------------------
// Exclusive scan: chunks of SCAN_IPB, block sums scanned recursively.
// ---------------------------------------------------------------------------
constexpr int SCAN_PER_THREAD = SCAN_IPB / SCAN_THREADS;

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_local(const T *in, T *out, int64_t n, T *bsum) {
    __shared__ T tile[SCAN_IPB];
    const int64_t base = (int64_t)blockIdx.x * SCAN_IPB;
    for (int k = threadIdx.x; k < SCAN_IPB; k += SCAN_THREADS) {
        int64_t idx = base + k;
        tile[k] = idx < n ? in[idx] : T(0);
    }
    __syncthreads();
    T v[SCAN_PER_THREAD];
    T s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        v[k] = tile[threadIdx.x * SCAN_PER_THREAD + k];
        s += v[k];
    }
    T total;
    T ex = block_exclusive_scan(s, &total);
#pragma unroll
    for (int k = 0; k < SCAN_PER_THREAD; ++k) {
        tile[threadIdx.x * SCAN_PER_THREAD + k] = ex;
        ex += v[k];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < SCAN_IPB; k += SCAN_THREADS) {
        int64_t idx = base + k;
        if (idx < n) out[idx] = tile[k];
    }
    if (threadIdx.x == 0 && bsum) bsum[blockIdx.x] = total;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_add(T *out, int64_t n, const T *boff) {
    const T add = boff[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * SCAN_IPB;
    for (int k = threadIdx.x; k < SCAN_IPB; k += SCAN_THREADS) {
        int64_t idx = base + k;
        if (idx < n) out[idx] += add;
    }
}

size_t scan_scratch_elems(int64_t n) {
    size_t total = 0;
    int64_t m = n;
    while (m > SCAN_IPB) {
        m = (m + SCAN_IPB - 1) / SCAN_IPB;
        total += (size_t)m + 64;
    }
    return total + 64;
}

template <typename T>
static cudaError_t scan_rec(const T *in, T *out, int64_t n, T *scratch, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int64_t nb = (n + SCAN_IPB - 1) / SCAN_IPB;
    if (nb == 1) {
        k_scan_local<T><<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr);
        note_launch();
        return cudaGetLastError();
    }
    T *sums = scratch;
    T *next = scratch + nb + 64;
    k_scan_local<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, sums);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_rec<T>(sums, sums, nb, next, s);
    if (e != cudaSuccess) return e;
    k_scan_add<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(out, n, sums);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *scratch, cudaStream_t s) {
    return scan_rec<uint32_t>(in, out, n, scratch, s);
}

cudaError_t launch_scan_u64(const unsigned long long *in, unsigned long long *out, int64_t n,
                            unsigned long long *scratch, cudaStream_t s) {
    return scan_rec<unsigned long long>(in, out, n, scratch, s);
}

// ---------------------------------------------------------------------------
// Segmented LSD radix sort.  The items of one call form contiguous segments
// (the views for the depth sort; the (plane, view) groups of the instances,
// which the emission writes in depth order) and each segment is sorted on
// its own: a block owns up to SORT_IPB consecutive items of one segment;
// the digit histogram of each segment is laid out [digit][block of the
// segment] after the earlier segments' histograms, so one device-wide
// exclusive scan yields every output position.  The digit of an item is
// taken from (key - key_base of its segment).
//
// Block-local ranking is stable and warp-private: warp w loads items
// [256 w, 256 w + 256) of the block into registers (eight coalesced rounds of
// 32) and ranks them with __match_any_sync against its own per-digit
// counters, then one block-wide pass turns the per-(warp, digit) counts into
// offsets.  Items are reordered in shared memory (16 KB a block) and written
// out coalesced.  The scatter is held to five resident blocks per SM: with
// more warps in flight it moves its bytes faster than the unbounded build
// (64 registers, four blocks), although the bound costs a few spilled words.
// ---------------------------------------------------------------------------
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_PER_WARP = SORT_IPB / SORT_WARPS;
constexpr int SORT_ROUNDS = SORT_PER_WARP / 32;
constexpr size_t SORT_SMEM = 2 * SORT_IPB * sizeof(uint32_t);

__device__ __forceinline__ int seg_of_block(const SegDev *segs, int nseg, int b) {
    return upper_index(nseg + 1, b, [&](int k) { return (int64_t)segs[k].blk_start; });
}

struct BlockSeg {
    uint32_t start, count, key_base;
    int32_t nb, lb;
    int64_t hbase;
};

// R: digit values of the pass (the histogram has R entries per block).
__device__ __forceinline__ bool block_seg(const SegDev *segs, int nseg, int b, BlockSeg &o, int R) {
    if ((uint32_t)b >= segs[nseg].blk_start) return false;  // sentinel holds the block total
    const int s = seg_of_block(segs, nseg, b);
    const SegDev sg = segs[s];
    o.lb = b - (int)sg.blk_start;
    o.nb = (int)((sg.len + SORT_IPB - 1) / SORT_IPB);
    o.start = sg.start + (uint32_t)o.lb * SORT_IPB;
    const uint32_t rem = sg.len - (uint32_t)o.lb * SORT_IPB;
    o.count = rem < (uint32_t)SORT_IPB ? rem : (uint32_t)SORT_IPB;
    o.key_base = sg.key_base;
    o.hbase = (int64_t)sg.blk_start * R;
    return true;
}

// Digit width BITS (4..8) per pass: the instance sort splits its key bits
// evenly over its passes, so no pass has more buckets than it needs (fewer
// buckets per block = longer coalesced runs in the scatter).
template <int BITS>
__global__ void __launch_bounds__(SORT_THREADS)
k_radix_hist(const uint32_t *__restrict__ keys, int shift, const SegDev *__restrict__ segs, int nseg,
             uint32_t *__restrict__ hist) {
    constexpr int R = 1 << BITS;
    __shared__ uint32_t cnt[R];
    BlockSeg bs;
    if (!block_seg(segs, nseg, blockIdx.x, bs, R)) return;
    for (int d = threadIdx.x; d < R; d += blockDim.x) cnt[d] = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < bs.count; i += blockDim.x)
        atomicAdd(&cnt[((keys[bs.start + i] - bs.key_base) >> shift) & (R - 1)], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < R; d += blockDim.x) hist[bs.hbase + (int64_t)d * bs.nb + bs.lb] = cnt[d];
}

template <int BITS>
__global__ void __launch_bounds__(SORT_THREADS, 5)
k_radix_scatter(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
                uint32_t *__restrict__ vout, int shift, const SegDev *__restrict__ segs, int nseg,
                const uint32_t *__restrict__ hscan) {
    constexpr int RADIX = 1 << BITS;  // digit values of this pass
    extern __shared__ uint32_t sm[];
    uint32_t *ok = sm, *ov = sm + SORT_IPB;
    __shared__ uint32_t wcnt[SORT_WARPS][RADIX];
    __shared__ uint32_t dstart[RADIX], gbase[RADIX];
    BlockSeg bs;
    if (!block_seg(segs, nseg, blockIdx.x, bs, RADIX)) return;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t n = bs.count;
    // this warp's items in registers (round r, lane l: item SORT_PER_WARP w + 32 r + l)
    uint32_t rk[SORT_ROUNDS], rv[SORT_ROUNDS];
#pragma unroll
    for (int r = 0; r < SORT_ROUNDS; ++r) {
        const uint32_t i = (uint32_t)(warp * SORT_PER_WARP + r * 32 + lane);
        rk[r] = i < n ? kin[bs.start + i] : 0u;
        rv[r] = i < n ? vin[bs.start + i] : 0u;
    }
    for (int d = t; d < RADIX; d += SORT_THREADS) {
#pragma unroll
        for (int w = 0; w < SORT_WARPS; ++w) wcnt[w][d] = 0;
    }
    __syncthreads();
    // warp-private stable ranking of this warp's 512 items
    const unsigned lt_mask = (1u << lane) - 1u;
    uint32_t lr[SORT_ROUNDS];
#pragma unroll
    for (int r = 0; r < SORT_ROUNDS; ++r) {
        const uint32_t i = (uint32_t)(warp * SORT_PER_WARP + r * 32 + lane);
        const bool valid = i < n;
        const uint32_t d = valid ? (((rk[r] - bs.key_base) >> shift) & (RADIX - 1)) : (uint32_t)RADIX;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const bool leader = (__ffs(peers) - 1) == lane;
        lr[r] = (valid ? wcnt[warp][d] : 0u) + (uint32_t)__popc(peers & lt_mask);
        __syncwarp();
        if (valid && leader) wcnt[warp][d] += (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: offsets of each warp, digit totals
    uint32_t tot = 0;
    if (t < RADIX) {
#pragma unroll
        for (int w = 0; w < SORT_WARPS; ++w) {
            const uint32_t c = wcnt[w][t];
            wcnt[w][t] = tot;
            tot += c;
        }
    }
    {
        const uint32_t ex = block_exclusive_scan<uint32_t>(t < RADIX ? tot : 0u, nullptr);
        if (t < RADIX) {
            dstart[t] = ex;
            gbase[t] = hscan[bs.hbase + (int64_t)t * bs.nb + bs.lb] - ex;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < SORT_ROUNDS; ++r) {
        const uint32_t i = (uint32_t)(warp * SORT_PER_WARP + r * 32 + lane);
        if (i < n) {
            const uint32_t k = rk[r];
            const uint32_t d = ((k - bs.key_base) >> shift) & (RADIX - 1);
            const uint32_t pos = dstart[d] + wcnt[warp][d] + lr[r];
            ok[pos] = k;
            ov[pos] = rv[r];
        }
    }
    __syncthreads();
    for (uint32_t p = t; p < n; p += SORT_THREADS) {
        const uint32_t k = ok[p];
        const uint32_t d = ((k - bs.key_base) >> shift) & (RADIX - 1);
        const uint32_t dst = gbase[d] + p;
        kout[dst] = k;
        vout[dst] = ov[p];
    }
}

// Single-block exclusive scan of the segments' block counts; entry nseg is a
// sentinel whose blk_start is the total.
__device__ void seg_blocks_scan(SegDev *segs, int nseg) {
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nseg; base += blockDim.x) {
        const int s = base + threadIdx.x;
        const uint32_t nb = s < nseg ? (segs[s].len + SORT_IPB - 1) / SORT_IPB : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan<uint32_t>(nb, &tot);
        if (s < nseg) segs[s].blk_start = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        segs[nseg].start = 0;
        segs[nseg].len = 0;
        segs[nseg].key_base = 0;
        segs[nseg].blk_start = carry;
    }
}

// Depth sort: one segment per view.
__global__ void __launch_bounds__(256) k_seg_views(const ViewDev *views, int V, SegDev *segs) {
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
        segs[v].start = (uint32_t)views[v].vg_off;
        segs[v].len = (uint32_t)views[v].N;
        segs[v].key_base = 0;
    }
    __syncthreads();
    seg_blocks_scan(segs, V);
}

// Instance sort: one segment per (plane, view); keys are global tile ids,
// key_base the segment's first tile.
__global__ void __launch_bounds__(256)
k_seg_instances(const unsigned long long *soff, const unsigned long long *scnt, int64_t VG, const ViewDev *views,
                int V, int tiles, const StatusDev *st, SegDev *segs) {
    const bool ok = st->code == SDGR_OK;
    const unsigned long long total = VG > 0 ? soff[2 * VG - 1] + scnt[2 * VG - 1] : 0ull;
    for (int s = threadIdx.x; s < 2 * V; s += blockDim.x) {
        const int p = s / V, v = s % V;
        const int64_t i0 = (int64_t)p * VG + views[v].vg_off;
        const unsigned long long a = i0 < 2 * VG ? soff[i0] : total;
        int64_t i1 = i0 + views[v].N;
        const unsigned long long b = i1 < 2 * VG ? soff[i1] : total;
        segs[s].start = (uint32_t)a;
        segs[s].len = ok ? (uint32_t)(b - a) : 0u;
        segs[s].key_base = (uint32_t)(p * tiles + views[v].tile_off);
    }
    __syncthreads();
    seg_blocks_scan(segs, 2 * V);
}

static bool g_sort_attr_done = false;

static cudaError_t sort_attrs() {
    if (g_sort_attr_done) return cudaSuccess;
    const int smem = (int)SORT_SMEM;
    cudaError_t e = cudaFuncSetAttribute(k_radix_scatter<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_radix_scatter<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_radix_scatter<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_radix_scatter<7>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_radix_scatter<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    g_sort_attr_done = true;
    return cudaSuccess;
}

template <int BITS>
static cudaError_t radix_pass(int nblocks, int nseg, const SegDev *segs, int shift, const uint32_t *kin,
                              const uint32_t *vin, uint32_t *kout, uint32_t *vout, uint32_t *hist,
                              uint32_t *scan_scratch, cudaStream_t s) {
    k_radix_hist<BITS><<<nblocks, SORT_THREADS, 0, s>>>(kin, shift, segs, nseg, hist);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = launch_scan_u32(hist, hist, (int64_t)nblocks * (1 << BITS), scan_scratch, s)) != cudaSuccess) return e;
    k_radix_scatter<BITS><<<nblocks, SORT_THREADS, SORT_SMEM, s>>>(kin, vin, kout, vout, shift, segs, nseg, hist);
    note_launch();
    return cudaGetLastError();
}

// LSD passes over the low `bits` bits: ceil(bits / 8) passes with the bits
// split evenly (at least 4 per pass).
static cudaError_t radix_passes(int nblocks, int nseg, const SegDev *segs, int bits, uint32_t *k0, uint32_t *v0,
                                uint32_t *k1, uint32_t *v1, uint32_t *hist, uint32_t *scan_scratch, int *passes_out,
                                cudaStream_t s) {
    cudaError_t e = sort_attrs();
    if (e != cudaSuccess) return e;
    uint32_t *kin = k0, *vin = v0, *kout = k1, *vout = v1;
    const int npass = bits <= 0 ? 0 : (bits + RADIX_BITS - 1) / RADIX_BITS;
    int digit = npass ? (bits + npass - 1) / npass : RADIX_BITS;
    if (digit < 4) digit = 4;
    int passes = 0;
    for (int shift = 0; passes < npass; shift += digit, ++passes) {
        switch (digit) {
            case 4: e = radix_pass<4>(nblocks, nseg, segs, shift, kin, vin, kout, vout, hist, scan_scratch, s); break;
            case 5: e = radix_pass<5>(nblocks, nseg, segs, shift, kin, vin, kout, vout, hist, scan_scratch, s); break;
            case 6: e = radix_pass<6>(nblocks, nseg, segs, shift, kin, vin, kout, vout, hist, scan_scratch, s); break;
            case 7: e = radix_pass<7>(nblocks, nseg, segs, shift, kin, vin, kout, vout, hist, scan_scratch, s); break;
            default: e = radix_pass<8>(nblocks, nseg, segs, shift, kin, vin, kout, vout, hist, scan_scratch, s); break;
        }
        if (e != cudaSuccess) return e;
        uint32_t *tk = kin, *tv = vin;
        kin = kout; vin = vout; kout = tk; vout = tv;
    }
    *passes_out = passes;
    return cudaSuccess;
}

cudaError_t launch_depth_sort(const ViewDev *views, int V, int nblocks, SegDev *segs, uint32_t *k0, uint32_t *v0,
                              uint32_t *k1, uint32_t *v1, uint32_t *hist, uint32_t *scan_scratch, cudaStream_t s) {
    if (nblocks <= 0 || V <= 0) return cudaSuccess;
    k_seg_views<<<1, 256, 0, s>>>(views, V, segs);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int passes = 0;
    return radix_passes(nblocks, V, segs, 32, k0, v0, k1, v1, hist, scan_scratch, &passes, s);
    // four passes: the result is back in (k0, v0)
}

cudaError_t launch_inst_sort(const StatusDev *st, const unsigned long long *soff, const unsigned long long *scnt,
                             int64_t VG, const ViewDev *views, int V, int tiles, int64_t cap, int key_bits,
                             SegDev *segs, uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, uint32_t *hist,
                             uint32_t *scan_scratch, int *final_in_1, cudaStream_t s) {
    *final_in_1 = 0;
    if (V <= 0) return cudaSuccess;
    const int nblocks = (int)((cap + SORT_IPB - 1) / SORT_IPB) + 2 * V;
    k_seg_instances<<<1, 256, 0, s>>>(soff, scnt, VG, views, V, tiles, st, segs);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int passes = 0;
    e = radix_passes(nblocks, 2 * V, segs, key_bits, k0, v0, k1, v1, hist, scan_scratch, &passes, s);
    *final_in_1 = passes & 1;
    return e;
}

// ---------------------------------------------------------------------------
// Instance counts in depth order, capacity check, emission, tile ranges.
// ---------------------------------------------------------------------------
__global__ void k_gather_counts(const uint32_t *__restrict__ sorted_vg, const BinRec *__restrict__ bin, int64_t VG,
                                unsigned long long *__restrict__ scnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < VG; k += stride) {
        const uint32_t vg = sorted_vg[k];
        const uint2 n = *reinterpret_cast<const uint2 *>(&bin[vg].nc);  // (nc, ni): one sector
        scnt[k] = n.x;
        scnt[VG + k] = n.y;
    }
}

cudaError_t launch_gather_counts(const uint32_t *sorted_vg, const BinRec *bin, int64_t VG, unsigned long long *scnt,
                                 int sms, cudaStream_t s) {
    if (VG <= 0) return cudaSuccess;
    int64_t blocks = (VG + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    k_gather_counts<<<(unsigned)blocks, 256, 0, s>>>(sorted_vg, bin, VG, scnt);
    note_launch();
    return cudaGetLastError();
}


// Position of the d-th (from 0) set bit of m; m has more than d set bits.
// Binary search over the low half of the remaining window: five steps.
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t m, uint32_t d) {
    uint32_t pos = 0u;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const uint32_t c = (uint32_t)__popc(m & ((1u << s) - 1u));
        if (d >= c) {
            d -= c;
            m >>= s;
            pos += (uint32_t)s;
        }
    }
    return pos;
}

__global__ void k_check_capacity(const unsigned long long *scnt, const unsigned long long *soff, int64_t VG,
                                 int64_t cap, StatusDev *st) {
    unsigned long long total = 0;
    if (VG > 0) total = soff[2 * VG - 1] + scnt[2 * VG - 1];
    st->required = (int64_t)total;
    if ((int64_t)total > cap) {
        st->code = SDGR_ERR_CAPACITY;
        st->n_inst = 0;
    } else {
        st->n_inst = (int64_t)total;
    }
}

cudaError_t launch_check_capacity(const unsigned long long *scnt, const unsigned long long *soff, int64_t VG,
                                  int64_t cap, StatusDev *st, cudaStream_t s) {
    k_check_capacity<<<1, 1, 0, s>>>(scnt, soff, VG, cap, st);
    note_launch();
    return cudaGetLastError();
}

// Instance emission, warp-cooperative: the 32 depth-sorted slots of a warp
// own one contiguous output range per plane (the counts' exclusive scan), and
// the warp writes that range with consecutive lanes on consecutive items.
// Item i belongs to the last lane whose range starts at or before i (five
// shuffle steps); inside a Gaussian's tile rectangle the items run row by row.
__global__ void __launch_bounds__(256)
k_emit(const uint32_t *__restrict__ sorted_vg, const unsigned long long *__restrict__ soff,
       const unsigned long long *__restrict__ scnt, const BinRec *__restrict__ bin,
       const ViewDev *__restrict__ views, int V, int64_t VG, int total_tiles, const StatusDev *st, int64_t cap,
       uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    if (st->code != SDGR_OK) return;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; k0 < VG; k0 += nwarps * 32) {
        const int64_t k = k0 + lane;
        const bool valid = k < VG;
        uint32_t vg = 0, tbase = 0;
        int tiles_x = 1;
        uint4 b0 = make_uint4(0u, 0u, 0u, 0u), b1 = make_uint4(0u, 0u, 0u, 0u);  // the slot's BinRec
        if (valid) {
            vg = sorted_vg[k];
            const uint4 *bp = reinterpret_cast<const uint4 *>(bin + vg);
            b0 = bp[0];
            b1 = bp[1];
            const ViewDev &vd = views[view_of_vg(views, V, k)];
            tiles_x = vd.tiles_x;
            tbase = (uint32_t)vd.tile_off;
        }
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const uint2 rect = p ? make_uint2(b0.z, b0.w) : make_uint2(b0.x, b0.y);
            const uint32_t tmask = p ? b1.y : b1.x;
            const unsigned long long off = valid ? soff[(int64_t)p * VG + k] : 0ull;
            const uint32_t cnt = valid ? (uint32_t)scnt[(int64_t)p * VG + k] : 0u;
            // rectangles of <= 32 tiles: ceil(2^16 / w), so that the row of a bit
            // index d < 32 is (d * rinv) >> 16 (exact: the error d (rinv - 2^16 / w) / 2^16
            // is below 32 / 2^16 < 1 / w); one division per Gaussian, none per instance
            uint32_t rinv = 0u;
            {
                const uint32_t tw = (rect.x >> 16) - (rect.x & 0xffffu) + 1u;
                const uint32_t th = (rect.y >> 16) - (rect.y & 0xffffu) + 1u;
                if (valid && cnt > 0u && tw * th <= 32u) rinv = (65536u + tw - 1u) / tw;
            }
            const unsigned long long off0 = __shfl_sync(full, off, 0);
            // start of this lane's range relative to lane 0 (an invalid lane
            // gets a start no item reaches)
            const uint32_t rel = valid ? (uint32_t)(off - off0) : 0xffffffffu;
            const uint32_t total = __reduce_max_sync(full, valid ? rel + cnt : 0u);
            const uint32_t key_base = (uint32_t)(p ? total_tiles : 0) + tbase;
            for (uint32_t i0 = 0; i0 < total; i0 += 32) {
                const uint32_t i = i0 + (uint32_t)lane;
                int o = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const uint32_t r2 = __shfl_sync(full, rel, (o + step) & 31);
                    if (o + step < 32 && r2 <= i) o += step;
                }
                const uint32_t o_rel = __shfl_sync(full, rel, o);
                const uint32_t o_rx = __shfl_sync(full, rect.x, o), o_ry = __shfl_sync(full, rect.y, o);
                const uint32_t o_mask = __shfl_sync(full, tmask, o);
                const uint32_t o_rinv = __shfl_sync(full, rinv, o);
                const uint32_t o_kb = __shfl_sync(full, key_base, o), o_vg = __shfl_sync(full, vg, o);
                const int o_tx = __shfl_sync(full, tiles_x, o);
                if (i < total) {
                    const uint32_t tx0 = o_rx & 0xffffu, w = (o_rx >> 16) - tx0 + 1u, ty0 = o_ry & 0xffffu;
                    const uint32_t h = (o_ry >> 16) - ty0 + 1u;
                    // the d-th tile of the Gaussian's set: of its rectangle, or
                    // the d-th set bit of its tile mask (rectangles of <= 32 tiles)
                    const bool small = w * h <= 32u;
                    const uint32_t d = small ? nth_set_bit(o_mask, i - o_rel) : i - o_rel;
                    const uint32_t q = small ? (d * o_rinv) >> 16 : d / w;
                    const uint32_t tx = tx0 + (d - q * w);
                    const unsigned long long pos = off0 + i;
                    if (SDGR_IN_BOUNDS(st, pos < (unsigned long long)cap)) {
                        keys[pos] = o_kb + (ty0 + q) * (uint32_t)o_tx + tx;
                        vals[pos] = o_vg;
                    }
                }
            }
        }
    }
    (void)cap;
}

cudaError_t launch_emit(const uint32_t *sorted_vg, const unsigned long long *soff, const unsigned long long *scnt,
                        const BinRec *bin, const ViewDev *views, int V, int64_t VG,
                        int total_tiles, const StatusDev *st, int64_t cap, uint32_t *keys, uint32_t *vals, int sms,
                        cudaStream_t s) {
    if (VG <= 0) return cudaSuccess;
    int64_t blocks = (VG + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    k_emit<<<(unsigned)blocks, 256, 0, s>>>(sorted_vg, soff, scnt, bin, views, V, VG, total_tiles, st, cap, keys,
                                            vals);
    note_launch();
    return cudaGetLastError();
}

// Each thread reads four consecutive keys as one 16-byte load (the key array
// starts 16-byte aligned) and the key on either side; a key that differs from
// its left (right) neighbour starts (ends) its range.
__global__ void k_ranges(const uint32_t *__restrict__ keys, StatusDev *st, int64_t cap, int64_t nranges,
                         uint2 *ranges) {
    int64_t n = st->code == SDGR_OK ? st->n_inst : 0;
    if (n > cap) n = cap;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n4 = (n + 3) / 4;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
        const int64_t i0 = 4 * q;
        uint32_t k[4];
        if (i0 + 3 < n) {
            const uint4 kv = *reinterpret_cast<const uint4 *>(keys + i0);
            k[0] = kv.x;
            k[1] = kv.y;
            k[2] = kv.z;
            k[3] = kv.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) k[e] = i0 + e < n ? keys[i0 + e] : 0u;
        }
        const uint32_t prev = i0 > 0 ? keys[i0 - 1] : 0u;
        const uint32_t next = i0 + 4 < n ? keys[i0 + 4] : 0u;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int64_t i = i0 + e;
            if (i >= n) break;
            if (!SDGR_IN_BOUNDS(st, (int64_t)k[e] < nranges)) continue;
            const uint32_t left = e == 0 ? prev : k[e - 1], right = e == 3 ? next : k[e + 1];
            if (i == 0 || left != k[e]) ranges[k[e]].x = (uint32_t)i;
            if (i == n - 1 || right != k[e]) ranges[k[e]].y = (uint32_t)(i + 1);
        }
    }
    (void)nranges;
}

cudaError_t launch_ranges(const uint32_t *keys, StatusDev *st, int64_t cap, int64_t nranges, uint2 *ranges, int sms,
                          cudaStream_t s) {
    int64_t blocks = (cap / 4 + 255) / 256;
    if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
    if (blocks < 1) blocks = 1;
    k_ranges<<<(unsigned)blocks, 256, 0, s>>>(keys, st, cap, nranges, ranges);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sdgr

namespace sdgr {

// ---------------------------------------------------------------------------
// Raster work lists.  Per plane: the tiles with a non-empty list, views in
// order, and inside each view in descending order of the bit length of the
// list size (a bucketed longest-processing-time order that keeps the tiles
// of one view -- and the records they share -- together on the GPU).
// Passes: per (plane, view, bucket) histogram; per (plane, view) totals;
// exclusive scan of the totals; per-view bucket offsets; scatter.  The
// order inside a bucket depends on atomic timing; a tile's result does not
// depend on when it runs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int order_bucket(uint2 r) { return 31 - __clz((int)(r.y - r.x)); }

__global__ void k_order_hist(const uint2 *__restrict__ ranges, int tiles, const ViewDev *__restrict__ views, int V,
                             uint32_t *vhist) {
    const int64_t n = 2 * (int64_t)tiles, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const uint2 r = ranges[k];
        if (r.y <= r.x) continue;
        const int p = k >= tiles;
        const int v = view_of_tile(views, V, k - (int64_t)p * tiles);
        atomicAdd(&vhist[((int64_t)p * V + v) * 32 + order_bucket(r)], 1u);
    }
}

__global__ void k_order_totals(const uint32_t *__restrict__ vhist, int V, uint32_t *vt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * (int64_t)V) return;
    uint32_t acc = 0;
    for (int b = 0; b < 32; ++b) acc += vhist[i * 32 + b];
    vt[i] = acc;
}

__global__ void k_order_offsets(const uint32_t *__restrict__ vhist, const uint32_t *__restrict__ vt,
                                const uint32_t *__restrict__ vbase, int V, uint32_t *voff, TileWorkDev *w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 2 * (int64_t)V) {
        const int p = i >= V;
        uint32_t acc = vbase[i] - (p ? vbase[V] : 0u);  // plane-local base
        for (int b = 31; b >= 0; --b) {
            voff[i * 32 + b] = acc;
            acc += vhist[i * 32 + b];
        }
    }
    if (i == 0) {
        w->count[0] = (int32_t)vbase[V];
        w->count[1] = (int32_t)(vbase[2 * V - 1] + vt[2 * V - 1] - vbase[V]);
        for (int k = 0; k < 4; ++k) w->next[k] = 0;
    }
}

__global__ void k_order_scatter(const uint2 *__restrict__ ranges, int tiles, const ViewDev *__restrict__ views, int V,
                                uint32_t *voff, int32_t *order) {
    const int64_t n = 2 * (int64_t)tiles, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const uint2 r = ranges[k];
        if (r.y <= r.x) continue;
        const int p = k >= tiles;
        const int64_t lt = k - (int64_t)p * tiles;
        const int v = view_of_tile(views, V, lt);
        const uint32_t slot = atomicAdd(&voff[((int64_t)p * V + v) * 32 + order_bucket(r)], 1u);
        order[(int64_t)p * tiles + slot] = (int32_t)lt;
    }
}

cudaError_t launch_tile_order(const uint2 *ranges, int tiles, const ViewDev *views, int V, TileWorkDev *work,
                              int32_t *order, uint32_t *vhist, uint32_t *voff, uint32_t *vt, uint32_t *vbase,
                              uint32_t *scratch, int sms, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(work, 0, sizeof(TileWorkDev), s);
    if (e != cudaSuccess || tiles <= 0 || V <= 0) return e;
    e = cudaMemsetAsync(vhist, 0, (size_t)2 * V * 32 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    int64_t blocks = (2 * (int64_t)tiles + 255) / 256;
    if (blocks > (int64_t)sms * 4) blocks = (int64_t)sms * 4;
    const unsigned vblocks = (unsigned)((2 * (int64_t)V + 255) / 256);
    k_order_hist<<<(unsigned)blocks, 256, 0, s>>>(ranges, tiles, views, V, vhist);
    note_launch();
    k_order_totals<<<vblocks, 256, 0, s>>>(vhist, V, vt);
    note_launch();
    e = launch_scan_u32(vt, vbase, 2 * (int64_t)V, scratch, s);
    if (e != cudaSuccess) return e;
    k_order_offsets<<<vblocks, 256, 0, s>>>(vhist, vt, vbase, V, voff, work);
    note_launch();
    k_order_scatter<<<(unsigned)blocks, 256, 0, s>>>(ranges, tiles, views, V, voff, order);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sdgr
