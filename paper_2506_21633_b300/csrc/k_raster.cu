// k_raster.cu -- steps a7, a8, a10, a11 of the rasterizer: the per-tile loops
// over depth-sorted Gaussians on the computation plane (scattering intensity,
// Section II-A-2, eq. I_i) and the layover splat on the imaging plane
// (Section II-A-3, eq. S_{n,m}), and their adjoints (Section II-B-1/2).
//
// One CTA per 16x16 tile, one thread per pixel (ray).  The tile's instance
// list is staged through shared memory in batches of 256 Gaussian records.
// Per-Gaussian sums over the tile's pixels are reduced across each warp with
// shuffles, then across warps in shared memory, then added to the
// per-(view, Gaussian) accumulators with one atomic per tile and Gaussian.
#include "sdgr_internal.cuh"

namespace sdgr {

constexpr int BATCH = 256;

struct TileCtx {
    int v;
    int px, py;
    bool inside;
    int64_t pix;
};

__device__ __forceinline__ TileCtx tile_ctx(const ViewDev *views, int V, int tile) {
    TileCtx c;
    c.v = view_of_tile(views, V, tile);
    const ViewDev &vd = views[c.v];
    const int lt = tile - vd.tile_off;
    const int tx = lt % vd.tiles_x, ty = lt / vd.tiles_x;
    c.px = tx * TILE + (threadIdx.x & (TILE - 1));
    c.py = ty * TILE + (threadIdx.x / TILE);
    c.inside = c.px < vd.NA && c.py < vd.NR;
    c.pix = vd.pix_off + (int64_t)c.py * vd.NA + c.px;
    return c;
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// ---------------------------------------------------------------------------
// a7: intensity pass.  Per ray (cell centre): T = 1; for each Gaussian in
// depth order: alpha = o exp(-delta/2) within the cutoff; the Gaussian
// receives alpha T; T *= 1 - alpha.  The ray stops once T < Tfloor.  For the
// adjoint each ray records the index just past its last in-cutoff Gaussian
// and the transmittance in front of that Gaussian.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_intensity_fwd(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals, const CompRec *__restrict__ comp,
                const ViewDev *__restrict__ views, int V, float cut, float Tfloor, const StatusDev *st,
                float *__restrict__ A, float *__restrict__ Tstop, int32_t *__restrict__ last) {
    if (st->code != SDGR_OK) return;
    __shared__ float4 sA[BATCH], sB[BATCH];
    __shared__ uint32_t sid[BATCH];
    __shared__ float sacc[BATCH];
    const int t = threadIdx.x, lane = t & 31;
    const TileCtx c = tile_ctx(views, V, blockIdx.x);
    const uint2 r = ranges[blockIdx.x];
    const float fx = (float)c.px, fy = (float)c.py;
    float T = 1.f, Tprev = 1.f;
    int32_t lastj = 0;
    bool done = !c.inside;
    for (uint32_t base = r.x; base < r.y; base += BATCH) {
        if (__syncthreads_count(done) == (int)blockDim.x) break;
        const uint32_t j = base + t;
        if (j < r.y) {
            const uint32_t vg = vals[j];
            const float4 *cp = reinterpret_cast<const float4 *>(comp + vg);
            sA[t] = cp[0];
            sB[t] = cp[1];
            sid[t] = vg;
        }
        sacc[t] = 0.f;
        __syncthreads();
        const int nb = min(BATCH, (int)(r.y - base));
        for (int k = 0; k < nb; ++k) {
            float contrib = 0.f;
            if (!done) {
                const float4 a = sA[k];
                const float4 b = sB[k];
                const float dx = __fsub_rn(fx, a.x), dy = __fsub_rn(fy, a.y);
                const float q = gauss_q(a.z, a.w, b.x, dx, dy);
                if (q >= cut) {
                    const float alpha = __fmul_rn(b.y, ex2_approx(q));
                    contrib = __fmul_rn(alpha, T);
                    Tprev = T;
                    lastj = (int32_t)(base + k + 1);
                    T = __fmul_rn(T, __fsub_rn(1.f, alpha));
                    if (T < Tfloor) done = true;
                }
            }
            if (__any_sync(0xffffffffu, contrib != 0.f)) {
                const float s = warp_sum(contrib);
                if (lane == 0 && s != 0.f) atomicAdd(&sacc[k], s);
            }
        }
        __syncthreads();
        if (t < nb && sacc[t] != 0.f) atomicAdd(&A[sid[t]], sacc[t]);
    }
    if (c.inside) {
        Tstop[c.pix] = Tprev;
        last[c.pix] = lastj;
    }
}

cudaError_t launch_intensity_fwd(const uint2 *ranges, const uint32_t *vals, const CompRec *comp, const ViewDev *views,
                                 int V, int tiles, float cut, float Tfloor, const StatusDev *st, float *A,
                                 float *Tstop, int32_t *last, cudaStream_t s) {
    if (tiles <= 0) return cudaSuccess;
    k_intensity_fwd<<<tiles, TILE_PIX, 0, s>>>(ranges, vals, comp, views, V, cut, Tfloor, st, A, Tstop, last);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a8: imaging splat.  S[pixel] = sum_i c_i exp(-delta_I/2) I_i, I_i = P_i A_i.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_splat_fwd(const uint2 *__restrict__ rangesI, const uint32_t *__restrict__ vals, const ImgRec *__restrict__ img,
            const CompRec *__restrict__ comp, const float *__restrict__ A, const ViewDev *__restrict__ views, int V,
            float cut, const StatusDev *st, float *__restrict__ images) {
    __shared__ float4 sA[BATCH];
    __shared__ float2 sB[BATCH];
    const int t = threadIdx.x;
    const TileCtx c = tile_ctx(views, V, blockIdx.x);
    const bool ok = st->code == SDGR_OK;
    const uint2 r = ok ? rangesI[blockIdx.x] : make_uint2(0u, 0u);
    const float fx = (float)c.px, fy = (float)c.py;
    float acc = 0.f;
    for (uint32_t base = r.x; base < r.y; base += BATCH) {
        __syncthreads();
        const uint32_t j = base + t;
        if (j < r.y) {
            const uint32_t vg = vals[j];
            const float4 *ip = reinterpret_cast<const float4 *>(img + vg);
            const float4 i0 = ip[0], i1 = ip[1];
            sA[t] = i0;
            sB[t] = make_float2(i1.x, i1.y * comp[vg].P * A[vg]);
        }
        __syncthreads();
        const int nb = min(BATCH, (int)(r.y - base));
        for (int k = 0; k < nb; ++k) {
            const float4 a = sA[k];
            const float2 b = sB[k];
            const float q = gauss_q(a.z, a.w, b.x, fx - a.x, fy - a.y);
            if (q >= cut) acc = fmaf(b.y, ex2_approx(q), acc);
        }
    }
    if (c.inside) images[c.pix] = acc;
}

cudaError_t launch_splat_fwd(const uint2 *rangesI, const uint32_t *vals, const ImgRec *img, const CompRec *comp,
                             const float *A, const ViewDev *views, int V, int tiles, float cut, const StatusDev *st,
                             float *images, cudaStream_t s) {
    if (tiles <= 0) return cudaSuccess;
    k_splat_fwd<<<tiles, TILE_PIX, 0, s>>>(rangesI, vals, img, comp, A, views, V, cut, st, images);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Shared-memory accumulation of six per-Gaussian moments of a per-pair
// weight w over the tile's pixels: sum w, w dx, w dy, w dx^2, w dx dy, w dy^2.
// ---------------------------------------------------------------------------
struct Moments {
    float m[6];
};

__device__ __forceinline__ void moments_of(float w, float dx, float dy, Moments &M) {
    const float wx = w * dx, wy = w * dy;
    M.m[0] = w;
    M.m[1] = wx;
    M.m[2] = wy;
    M.m[3] = wx * dx;
    M.m[4] = wx * dy;
    M.m[5] = wy * dy;
}

__device__ __forceinline__ void reduce_moments(Moments &M, bool any, int lane, float (*sacc)[BATCH], int k) {
    if (__any_sync(0xffffffffu, any)) {
#pragma unroll
        for (int q = 0; q < 6; ++q) M.m[q] = warp_sum(M.m[q]);
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < 6; ++q)
                if (M.m[q] != 0.f) atomicAdd(&sacc[q][k], M.m[q]);
        }
    }
}

__device__ __forceinline__ void flush_moments(float (*sacc)[BATCH], int t, uint32_t vg, float4 *acc) {
    const float a0 = sacc[0][t], a1 = sacc[1][t], a2 = sacc[2][t], a3 = sacc[3][t], a4 = sacc[4][t],
                a5 = sacc[5][t];
    if (a0 != 0.f || a1 != 0.f || a2 != 0.f || a3 != 0.f || a4 != 0.f || a5 != 0.f) {
        float *p = reinterpret_cast<float *>(acc + 2 * (size_t)vg);
        atomicAdd(p + 0, a0);
        atomicAdd(p + 1, a1);
        atomicAdd(p + 2, a2);
        atomicAdd(p + 3, a3);
        atomicAdd(p + 4, a4);
        atomicAdd(p + 5, a5);
    }
}

// ---------------------------------------------------------------------------
// a10: adjoint of the imaging splat.  Per (view, Gaussian) the moments of
// w = dL/dS * exp(-delta_I/2); the parameter adjoint turns them into
// dL/dI = c M0, dL/du_I, dL/dconic_I and dL/dc.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_splat_bwd(const uint2 *__restrict__ rangesI, const uint32_t *__restrict__ vals, const ImgRec *__restrict__ img,
            const float *__restrict__ dLdS, const ViewDev *__restrict__ views, int V, float cut, const StatusDev *st,
            float4 *__restrict__ accI) {
    if (st->code != SDGR_OK) return;
    __shared__ float4 sA[BATCH];
    __shared__ float sC[BATCH];
    __shared__ uint32_t sid[BATCH];
    __shared__ float sacc[6][BATCH];
    const int t = threadIdx.x, lane = t & 31;
    const TileCtx c = tile_ctx(views, V, blockIdx.x);
    const uint2 r = rangesI[blockIdx.x];
    const float fx = (float)c.px, fy = (float)c.py;
    const float g = c.inside ? dLdS[c.pix] : 0.f;
    if (__syncthreads_count(g != 0.f) == 0) return;
    for (uint32_t base = r.x; base < r.y; base += BATCH) {
        __syncthreads();
        const uint32_t j = base + t;
        if (j < r.y) {
            const uint32_t vg = vals[j];
            const float4 *ip = reinterpret_cast<const float4 *>(img + vg);
            sA[t] = ip[0];
            sC[t] = ip[1].x;
            sid[t] = vg;
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) sacc[q][t] = 0.f;
        __syncthreads();
        const int nb = min(BATCH, (int)(r.y - base));
        for (int k = 0; k < nb; ++k) {
            const float4 a = sA[k];
            const float dx = fx - a.x, dy = fy - a.y;
            const float q = gauss_q(a.z, a.w, sC[k], dx, dy);
            Moments M;
            const bool hit = q >= cut && g != 0.f;
            moments_of(hit ? g * ex2_approx(q) : 0.f, dx, dy, M);
            reduce_moments(M, hit, lane, sacc, k);
        }
        __syncthreads();
        if (t < nb) flush_moments(sacc, t, sid[t], accI);
    }
}

cudaError_t launch_splat_bwd(const uint2 *rangesI, const uint32_t *vals, const ImgRec *img, const float *dLdS,
                             const ViewDev *views, int V, int tiles, float cut, const StatusDev *st, float4 *accI,
                             cudaStream_t s) {
    if (tiles <= 0) return cudaSuccess;
    k_splat_bwd<<<tiles, TILE_PIX, 0, s>>>(rangesI, vals, img, dLdS, views, V, cut, st, accI);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a11: adjoint of the intensity pass.  With chat_i = dL/dI_i P_i the ray's
// share of L is sum_i chat_i alpha_i T_i, so dL/dalpha_i = T_i (chat_i - B_i),
// B_i = sum_{j>i} chat_j alpha_j prod_{i<k<j}(1 - alpha_k).  Each ray walks
// its list back to front from the last in-cutoff Gaussian the forward pass
// recorded: B by the suffix recursion B <- chat alpha + (1 - alpha) B, T by
// undoing the forward products (T_i = T_{i+1} / (1 - alpha_i), with the same
// float bits of alpha; every factor is > 0 because T_{i+1} >= Tfloor).
// Per (view, Gaussian) the moments of w = dL/dalpha exp(-delta_C/2).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_intensity_bwd(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals, const CompRec *__restrict__ comp,
                const ImgRec *__restrict__ img, const float4 *__restrict__ accI, const float *__restrict__ Tstop,
                const int32_t *__restrict__ last, const ViewDev *__restrict__ views, int V, float cut,
                const StatusDev *st, float4 *__restrict__ accC) {
    if (st->code != SDGR_OK) return;
    __shared__ float4 sA[BATCH], sB[BATCH];
    __shared__ uint32_t sid[BATCH];
    __shared__ float sacc[6][BATCH];
    __shared__ int smax;
    const int t = threadIdx.x, lane = t & 31;
    const TileCtx c = tile_ctx(views, V, blockIdx.x);
    const uint2 r = ranges[blockIdx.x];
    const float fx = (float)c.px, fy = (float)c.py;
    const int32_t mylast = c.inside ? last[c.pix] : 0;
    float T = c.inside ? Tstop[c.pix] : 0.f;
    if (t == 0) smax = 0;
    __syncthreads();
    if (mylast > 0) atomicMax(&smax, mylast);
    __syncthreads();
    const int hi0 = smax;
    float B = 0.f;
    bool first = true;
    for (int hi = hi0; hi > (int)r.x; hi -= BATCH) {
        const int lo = max((int)r.x, hi - BATCH);
        const int nb = hi - lo;
        __syncthreads();
        if (t < nb) {
            const uint32_t vg = vals[lo + t];
            const float4 *cp = reinterpret_cast<const float4 *>(comp + vg);
            const float4 c0 = cp[0], c1 = cp[1];
            const float dLdI = accI[2 * (size_t)vg].x * img[vg].cn;
            sA[t] = c0;
            sB[t] = make_float4(c1.x, c1.y, dLdI * c1.z, 0.f);
            sid[t] = vg;
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) sacc[q][t] = 0.f;
        __syncthreads();
        for (int k = nb - 1; k >= 0; --k) {
            const int j = lo + k;
            float w = 0.f, dx = 0.f, dy = 0.f;
            bool hit = false;
            if (j < mylast) {
                const float4 a = sA[k];
                const float4 b = sB[k];
                dx = __fsub_rn(fx, a.x);
                dy = __fsub_rn(fy, a.y);
                const float q = gauss_q(a.z, a.w, b.x, dx, dy);
                if (q >= cut) {
                    const float e = ex2_approx(q);
                    const float alpha = __fmul_rn(b.y, e);
                    if (!first) T = __fdiv_rn(T, __fsub_rn(1.f, alpha));
                    first = false;
                    const float chat = b.z;
                    const float ga = T * (chat - B);
                    B = fmaf(chat, alpha, (1.f - alpha) * B);
                    w = ga * e;
                    hit = true;
                }
            }
            Moments M;
            moments_of(w, dx, dy, M);
            reduce_moments(M, hit, lane, sacc, k);
        }
        __syncthreads();
        if (t < nb) flush_moments(sacc, t, sid[t], accC);
    }
}

cudaError_t launch_intensity_bwd(const uint2 *ranges, const uint32_t *vals, const CompRec *comp, const ImgRec *img,
                                 const float4 *accI, const float *Tstop, const int32_t *last, const ViewDev *views,
                                 int V, int tiles, float cut, const StatusDev *st, float4 *accC, cudaStream_t s) {
    if (tiles <= 0) return cudaSuccess;
    k_intensity_bwd<<<tiles, TILE_PIX, 0, s>>>(ranges, vals, comp, img, accI, Tstop, last, views, V, cut, st, accC);
    note_launch();
    return cudaGetLastError();
}

// Diagnostic: in-cutoff (pixel, Gaussian) pairs of every tile of one plane.
template <typename Rec>
__global__ void __launch_bounds__(256)
k_count_pairs(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals, const Rec *__restrict__ rec,
              const ViewDev *__restrict__ views, int V, float cut, unsigned long long *out) {
    __shared__ float4 sA[BATCH];
    __shared__ float sC[BATCH];
    const int t = threadIdx.x;
    const TileCtx c = tile_ctx(views, V, blockIdx.x);
    const uint2 r = ranges[blockIdx.x];
    const float fx = (float)c.px, fy = (float)c.py;
    unsigned int n = 0;
    for (uint32_t base = r.x; base < r.y; base += BATCH) {
        __syncthreads();
        const uint32_t j = base + t;
        if (j < r.y) {
            const float4 *p = reinterpret_cast<const float4 *>(rec + vals[j]);
            sA[t] = p[0];
            sC[t] = p[1].x;
        }
        __syncthreads();
        const int nb = min(BATCH, (int)(r.y - base));
        if (c.inside)
            for (int k = 0; k < nb; ++k) {
                const float4 a = sA[k];
                n += gauss_q(a.z, a.w, sC[k], __fsub_rn(fx, a.x), __fsub_rn(fy, a.y)) >= cut;
            }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((t & 31) == 0 && n) atomicAdd(out, (unsigned long long)n);
}

cudaError_t launch_count_pairs(const uint2 *ranges, const uint32_t *vals, const CompRec *comp, const ImgRec *img,
                               const ViewDev *views, int V, int tiles, float cut, StatusDev *st, cudaStream_t s) {
    if (tiles <= 0) return cudaSuccess;
    k_count_pairs<CompRec><<<tiles, TILE_PIX, 0, s>>>(ranges, vals, comp, views, V, cut, &st->pairs[0]);
    note_launch();
    k_count_pairs<ImgRec><<<tiles, TILE_PIX, 0, s>>>(ranges + tiles, vals, img, views, V, cut, &st->pairs[1]);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_intensity_out(const CompRec *__restrict__ comp, const float *__restrict__ A, int64_t VG,
                                float *__restrict__ I) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < VG; i += stride) I[i] = comp[i].P * A[i];
}

cudaError_t launch_intensity_out(const CompRec *comp, const float *A, int64_t VG, float *I, int sms, cudaStream_t s) {
    if (VG <= 0) return cudaSuccess;
    int64_t blocks = (VG + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    k_intensity_out<<<(unsigned)blocks, 256, 0, s>>>(comp, A, VG, I);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sdgr
