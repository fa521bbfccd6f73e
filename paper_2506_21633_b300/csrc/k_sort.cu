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
// LSD radix sort passes.  A block owns SORT_IPB consecutive items of one
// segment.  Segmented mode (depth sort): segments are views, block -> view
// by the per-view block offsets; the digit histogram of each view is laid out
// [digit][block of the view] after the earlier views' histograms, so one
// device-wide exclusive scan yields every output position.  Single mode
// (instance sort): one segment whose length is read on the device.
// ---------------------------------------------------------------------------
struct Seg {
    int64_t start;
    int32_t count;
    int32_t nb, lb;
    int64_t hbase;
};

template <bool VIEWS>
__device__ __forceinline__ Seg seg_of(int b, const ViewDev *views, int V, const StatusDev *st, int64_t cap,
                                      int nblocks) {
    Seg s;
    if (VIEWS) {
        const int v = view_of_sblk(views, V, b);
        const ViewDev &vd = views[v];
        s.lb = b - vd.sblk_off;
        s.nb = vd.sblk_n;
        s.start = vd.vg_off + (int64_t)s.lb * SORT_IPB;
        int64_t rem = (int64_t)vd.N - (int64_t)s.lb * SORT_IPB;
        s.count = (int32_t)(rem < SORT_IPB ? (rem > 0 ? rem : 0) : SORT_IPB);
        s.hbase = (int64_t)vd.sblk_off * RADIX;
    } else {
        int64_t n = st->code == SDGR_OK ? st->n_inst : 0;
        if (n > cap) n = cap;
        s.lb = b;
        s.nb = nblocks;
        s.start = (int64_t)b * SORT_IPB;
        int64_t rem = n - s.start;
        s.count = (int32_t)(rem < SORT_IPB ? (rem > 0 ? rem : 0) : SORT_IPB);
        s.hbase = 0;
    }
    return s;
}

template <bool VIEWS>
__global__ void __launch_bounds__(SORT_THREADS)
k_radix_hist(const uint32_t *__restrict__ keys, int shift, const ViewDev *views, int V, const StatusDev *st,
             int64_t cap, int nblocks, uint32_t *__restrict__ hist) {
    __shared__ uint32_t cnt[RADIX];
    const Seg sg = seg_of<VIEWS>(blockIdx.x, views, V, st, cap, nblocks);
    for (int d = threadIdx.x; d < RADIX; d += blockDim.x) cnt[d] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < sg.count; i += blockDim.x)
        atomicAdd(&cnt[(keys[sg.start + i] >> shift) & (RADIX - 1)], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < RADIX; d += blockDim.x) hist[sg.hbase + (int64_t)d * sg.nb + sg.lb] = cnt[d];
}

constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr size_t SORT_SMEM = 4 * SORT_IPB * sizeof(uint32_t);

template <bool VIEWS>
__global__ void __launch_bounds__(SORT_THREADS)
k_radix_scatter(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
                uint32_t *__restrict__ vout, int shift, const ViewDev *views, int V, const StatusDev *st, int64_t cap,
                int nblocks, const uint32_t *__restrict__ hscan) {
    extern __shared__ uint32_t sm[];
    uint32_t *sk = sm, *sv = sm + SORT_IPB, *ok = sm + 2 * SORT_IPB, *ov = sm + 3 * SORT_IPB;
    __shared__ uint32_t cnt[RADIX], lstart[RADIX], run[RADIX], gbase[RADIX];
    __shared__ uint32_t wcnt[SORT_WARPS][RADIX];

    const Seg sg = seg_of<VIEWS>(blockIdx.x, views, V, st, cap, nblocks);
    if (sg.count == 0) return;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int i = t; i < sg.count; i += SORT_THREADS) {
        sk[i] = kin[sg.start + i];
        sv[i] = vin[sg.start + i];
    }
    for (int d = t; d < RADIX; d += SORT_THREADS) {
        cnt[d] = 0;
        run[d] = 0;
#pragma unroll
        for (int w = 0; w < SORT_WARPS; ++w) wcnt[w][d] = 0;
    }
    __syncthreads();
    for (int i = t; i < sg.count; i += SORT_THREADS) atomicAdd(&cnt[(sk[i] >> shift) & (RADIX - 1)], 1u);
    __syncthreads();
    {
        uint32_t c = t < RADIX ? cnt[t] : 0u;
        uint32_t ex = block_exclusive_scan<uint32_t>(c, nullptr);
        if (t < RADIX) {
            lstart[t] = ex;
            gbase[t] = hscan[sg.hbase + (int64_t)t * sg.nb + sg.lb] - ex;
        }
    }
    __syncthreads();
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int r0 = 0; r0 < sg.count; r0 += SORT_THREADS) {
        const int i = r0 + t;
        const bool valid = i < sg.count;
        const uint32_t d = valid ? ((sk[i] >> shift) & (RADIX - 1)) : (uint32_t)RADIX;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & lt_mask);
        const bool leader = (__ffs(peers) - 1) == lane;
        if (valid && leader) wcnt[warp][d] = (uint32_t)__popc(peers);
        __syncthreads();
        if (t < RADIX) {
            uint32_t acc = run[t];
#pragma unroll
            for (int w = 0; w < SORT_WARPS; ++w) {
                uint32_t c = wcnt[w][t];
                wcnt[w][t] = acc;
                acc += c;
            }
            run[t] = acc;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = lstart[d] + wcnt[warp][d] + rank;
            ok[pos] = sk[i];
            ov[pos] = sv[i];
        }
        __syncthreads();
        if (t < RADIX) {
#pragma unroll
            for (int w = 0; w < SORT_WARPS; ++w) wcnt[w][t] = 0;
        }
        __syncthreads();
    }
    for (int p = t; p < sg.count; p += SORT_THREADS) {
        const uint32_t k = ok[p];
        const uint32_t d = (k >> shift) & (RADIX - 1);
        const uint32_t dst = gbase[d] + (uint32_t)p;
        kout[dst] = k;
        vout[dst] = ov[p];
    }
}

static bool g_sort_attr_done = false;

static cudaError_t sort_attrs() {
    if (g_sort_attr_done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_radix_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SORT_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_radix_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SORT_SMEM);
    if (e != cudaSuccess) return e;
    g_sort_attr_done = true;
    return cudaSuccess;
}

cudaError_t launch_depth_sort(const ViewDev *views, int V, int nblocks, uint32_t *k0, uint32_t *v0, uint32_t *k1,
                              uint32_t *v1, uint32_t *hist, uint32_t *scan_scratch, cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    cudaError_t e = sort_attrs();
    if (e != cudaSuccess) return e;
    uint32_t *kin = k0, *vin = v0, *kout = k1, *vout = v1;
    const int64_t hn = (int64_t)nblocks * RADIX;
    for (int shift = 0; shift < 32; shift += RADIX_BITS) {
        k_radix_hist<true><<<nblocks, SORT_THREADS, 0, s>>>(kin, shift, views, V, nullptr, 0, nblocks, hist);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = launch_scan_u32(hist, hist, hn, scan_scratch, s)) != cudaSuccess) return e;
        k_radix_scatter<true><<<nblocks, SORT_THREADS, SORT_SMEM, s>>>(kin, vin, kout, vout, shift, views, V, nullptr,
                                                                      0, nblocks, hist);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        uint32_t *tk = kin, *tv = vin;
        kin = kout; vin = vout; kout = tk; vout = tv;
    }
    return cudaSuccess;  // four passes: the result is back in (k0, v0)
}

cudaError_t launch_inst_sort(const StatusDev *st, int64_t cap, int key_bits, uint32_t *k0, uint32_t *v0,
                             uint32_t *k1, uint32_t *v1, uint32_t *hist, uint32_t *scan_scratch, int *final_in_1,
                             cudaStream_t s) {
    *final_in_1 = 0;
    const int nblocks = (int)((cap + SORT_IPB - 1) / SORT_IPB);
    if (nblocks <= 0) return cudaSuccess;
    cudaError_t e = sort_attrs();
    if (e != cudaSuccess) return e;
    uint32_t *kin = k0, *vin = v0, *kout = k1, *vout = v1;
    const int64_t hn = (int64_t)nblocks * RADIX;
    int passes = 0;
    for (int shift = 0; shift < key_bits; shift += RADIX_BITS, ++passes) {
        k_radix_hist<false><<<nblocks, SORT_THREADS, 0, s>>>(kin, shift, nullptr, 0, st, cap, nblocks, hist);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = launch_scan_u32(hist, hist, hn, scan_scratch, s)) != cudaSuccess) return e;
        k_radix_scatter<false><<<nblocks, SORT_THREADS, SORT_SMEM, s>>>(kin, vin, kout, vout, shift, nullptr, 0, st,
                                                                       cap, nblocks, hist);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        uint32_t *tk = kin, *tv = vin;
        kin = kout; vin = vout; kout = tk; vout = tv;
    }
    *final_in_1 = passes & 1;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Instance counts in depth order, capacity check, emission, tile ranges.
// ---------------------------------------------------------------------------
__global__ void k_gather_counts(const uint32_t *__restrict__ sorted_vg, const uint32_t *__restrict__ cntC,
                                const uint32_t *__restrict__ cntI, int64_t VG, unsigned long long *__restrict__ scnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < VG; k += stride) {
        const uint32_t vg = sorted_vg[k];
        scnt[k] = cntC[vg];
        scnt[VG + k] = cntI[vg];
    }
}

cudaError_t launch_gather_counts(const uint32_t *sorted_vg, const uint32_t *cntC, const uint32_t *cntI, int64_t VG,
                                 unsigned long long *scnt, int sms, cudaStream_t s) {
    if (VG <= 0) return cudaSuccess;
    int64_t blocks = (VG + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    k_gather_counts<<<(unsigned)blocks, 256, 0, s>>>(sorted_vg, cntC, cntI, VG, scnt);
    note_launch();
    return cudaGetLastError();
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

__device__ __forceinline__ void emit_rect(uint2 rect, unsigned long long base, uint32_t tile_base, int tiles_x,
                                          uint32_t vg, uint32_t *keys, uint32_t *vals) {
    const int tx0 = rect.x & 0xffff, tx1 = rect.x >> 16, ty0 = rect.y & 0xffff, ty1 = rect.y >> 16;
    unsigned long long p = base;
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) {
            keys[p] = tile_base + (uint32_t)(ty * tiles_x + tx);
            vals[p] = vg;
            ++p;
        }
}

__global__ void __launch_bounds__(256)
k_emit(const uint32_t *__restrict__ sorted_vg, const unsigned long long *__restrict__ soff,
       const uint2 *__restrict__ rectC, const uint2 *__restrict__ rectI, const ViewDev *__restrict__ views, int V,
       int64_t VG, int total_tiles, const StatusDev *st, uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    if (st->code != SDGR_OK) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < VG; k += stride) {
        const uint32_t vg = sorted_vg[k];
        const int v = view_of_vg(views, V, k);
        const ViewDev &vd = views[v];
        const uint2 rc = rectC[vg];
        if (rc.x != 0xffffffffu) emit_rect(rc, soff[k], (uint32_t)vd.tile_off, vd.tiles_x, vg, keys, vals);
        const uint2 ri = rectI[vg];
        if (ri.x != 0xffffffffu)
            emit_rect(ri, soff[VG + k], (uint32_t)(total_tiles + vd.tile_off), vd.tiles_x, vg, keys, vals);
    }
}

cudaError_t launch_emit(const uint32_t *sorted_vg, const unsigned long long *soff, const uint2 *rectC,
                        const uint2 *rectI, const ViewDev *views, int V, int64_t VG, int total_tiles,
                        const StatusDev *st, uint32_t *keys, uint32_t *vals, int sms, cudaStream_t s) {
    if (VG <= 0) return cudaSuccess;
    int64_t blocks = (VG + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    k_emit<<<(unsigned)blocks, 256, 0, s>>>(sorted_vg, soff, rectC, rectI, views, V, VG, total_tiles, st, keys, vals);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_ranges(const uint32_t *__restrict__ keys, const StatusDev *st, int64_t cap, uint2 *ranges) {
    int64_t n = st->code == SDGR_OK ? st->n_inst : 0;
    if (n > cap) n = cap;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t k = keys[i];
        if (i == 0 || keys[i - 1] != k) ranges[k].x = (uint32_t)i;
        if (i == n - 1 || keys[i + 1] != k) ranges[k].y = (uint32_t)(i + 1);
    }
}

cudaError_t launch_ranges(const uint32_t *keys, const StatusDev *st, int64_t cap, uint2 *ranges, int sms,
                          cudaStream_t s) {
    int64_t blocks = (cap + 255) / 256;
    if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
    if (blocks < 1) blocks = 1;
    k_ranges<<<(unsigned)blocks, 256, 0, s>>>(keys, st, cap, ranges);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sdgr
