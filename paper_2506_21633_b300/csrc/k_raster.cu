// k_raster.cu -- steps a7, a8, a10, a11 of the rasterizer: the per-tile loops
// over depth-sorted Gaussians on the computation plane (scattering intensity,
// Section II-A-2, eq. I_i) and the layover splat on the imaging plane
// (Section II-A-3, eq. S_{n,m}), and their adjoints (Section II-B-1/2).
//
// One CTA per 16x16 tile, one thread per pixel (ray).  The tile's instance
// list is staged through shared memory in batches of 256 Gaussian records.
//
// Sums over the tile's pixels per Gaussian (the ray sums A_i of the intensity
// pass and the six moments of the adjoints) use a two-phase transpose
// instead of warp-shuffle reductions: in phase 1 every thread (pixel) walks a
// sub-batch of 32 Gaussians in list order and writes each pair's weight into
// a 32 x 256 shared-memory table; in phase 2 eight threads per Gaussian sum
// that Gaussian's row of the table (two columns each, only over the rows its
// K-ellipse can reach), and three shuffles combine the eight partial sums.
// The table's row stride (264 floats) makes both the phase-1 stores and the
// phase-2 loads free of bank conflicts.  A warp (two pixel rows) skips a
// Gaussian whose K-ellipse misses both of its rows.
#include "sdgr_internal.cuh"

namespace sdgr {

constexpr int BATCH = 256;    // Gaussian records staged per batch
constexpr int SUB = 32;       // Gaussians per weight table
constexpr int WSTRIDE = 264;  // row stride of the weight table (floats)

struct TileCtx {
    int v;
    int x0, y0;  // pixel coordinates of the tile's first pixel
    int px, py;  // this thread's pixel
    bool inside;
    int64_t pix;
};

__device__ __forceinline__ TileCtx tile_ctx(const ViewDev *views, int V, int tile) {
    TileCtx c;
    c.v = view_of_tile(views, V, tile);
    const ViewDev &vd = views[c.v];
    const int lt = tile - vd.tile_off;
    c.x0 = (lt % vd.tiles_x) * TILE;
    c.y0 = (lt / vd.tiles_x) * TILE;
    c.px = c.x0 + (threadIdx.x & (TILE - 1));
    c.py = c.y0 + (threadIdx.x / TILE);
    c.inside = c.px < vd.NA && c.py < vd.NR;
    c.pix = vd.pix_off + (int64_t)c.py * vd.NA + c.px;
    return c;
}

// Tile-local rows [x, y] that the K-ellipse of a Gaussian centred at row uy
// with bounding-box half-height ry can reach (empty when x > y).
__device__ __forceinline__ int2 tile_rows(float uy, float ry, int y0) {
    float lo = ceilf(uy - ry) - (float)y0, hi = floorf(uy + ry) - (float)y0;
    lo = fminf(fmaxf(lo, 0.f), 16.f);
    hi = fminf(fmaxf(hi, -1.f), 15.f);
    if (!(lo <= 16.f)) lo = 0.f;  // NaN centre: keep every row, the pair test decides
    if (!(hi >= -1.f)) hi = 15.f;
    return make_int2((int)lo, (int)hi);
}

// Does the ellipse reach either of the two rows of warp w?
__device__ __forceinline__ bool warp_rows_hit(int2 rows, int warp) {
    return rows.y >= 2 * warp && rows.x <= 2 * warp + 1;
}

// Phase 2, one sum: every lane of the group of eight returns the sum of
// Gaussian (threadIdx.x / 8)'s table row over the rows [rows.x, rows.y].
__device__ __forceinline__ float table_sum(const float *W, int2 rows) {
    const int j = threadIdx.x >> 3, c = threadIdx.x & 7;
    const float *w = W + j * WSTRIDE + c;
    float s = 0.f;
    for (int r = rows.x; r <= rows.y; ++r) s += w[r * TILE] + w[r * TILE + 8];
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    return s;
}

// Phase 2, six moments of the weights w over the pixels: sum w, w dx, w dy,
// w dx^2, w dx dy, w dy^2 with (dx, dy) = pixel - centre.  dx0 = offset of
// the thread's first column (x0 + c - ux), dy0 = y0 - uy.
__device__ __forceinline__ void table_moments(const float *W, int2 rows, float dx0, float dy0, float m[6]) {
    const int j = threadIdx.x >> 3, c = threadIdx.x & 7;
    const float *w = W + j * WSTRIDE + c;
    const float dx1 = dx0 + 8.f;
    float m0 = 0.f, mx = 0.f, my = 0.f, mxx = 0.f, mxy = 0.f, myy = 0.f;
    for (int r = rows.x; r <= rows.y; ++r) {
        const float dy = dy0 + (float)r;
        const float w0 = w[r * TILE], w1 = w[r * TILE + 8];
        const float a0 = w0 * dx0, a1 = w1 * dx1;
        const float ws = w0 + w1, as = a0 + a1;
        m0 += ws;
        mx += as;
        my = fmaf(ws, dy, my);
        mxx = fmaf(a0, dx0, fmaf(a1, dx1, mxx));
        mxy = fmaf(as, dy, mxy);
        myy = fmaf(ws * dy, dy, myy);
    }
    m[0] = m0; m[1] = mx; m[2] = my; m[3] = mxx; m[4] = mxy; m[5] = myy;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        m[q] += __shfl_xor_sync(0xffffffffu, m[q], 1);
        m[q] += __shfl_xor_sync(0xffffffffu, m[q], 2);
        m[q] += __shfl_xor_sync(0xffffffffu, m[q], 4);
    }
}

__device__ __forceinline__ void add_moments(float4 *acc, uint32_t vg, const float m[6]) {
    if (m[0] != 0.f || m[1] != 0.f || m[2] != 0.f || m[3] != 0.f || m[4] != 0.f || m[5] != 0.f) {
        float *p = reinterpret_cast<float *>(acc + 2 * (size_t)vg);
#pragma unroll
        for (int q = 0; q < 6; ++q) atomicAdd(p + q, m[q]);
    }
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
    __shared__ float4 sA[BATCH];
    __shared__ float2 sB[BATCH];
    __shared__ int2 sR[BATCH];
    __shared__ uint32_t sid[BATCH];
    __shared__ float W[SUB * WSTRIDE];
    const int t = threadIdx.x, warp = t >> 5;
    const TileCtx c = tile_ctx(views, V, blockIdx.x);
    const uint2 r = ranges[blockIdx.x];
    const float fx = (float)c.px, fy = (float)c.py;
    float T = 1.f, Tprev = 1.f;
    int32_t lastj = 0;
    bool done = !c.inside;
    for (uint32_t base = r.x; base < r.y; base += BATCH) {
        if (__syncthreads_count(done) == (int)blockDim.x) break;
        const uint32_t jload = base + t;
        if (jload < r.y) {
            const uint32_t vg = vals[jload];
            const float4 *cp = reinterpret_cast<const float4 *>(comp + vg);
            const float4 c0 = cp[0], c1 = cp[1];
            sA[t] = c0;
            sB[t] = make_float2(c1.x, c1.y);
            sR[t] = tile_rows(c0.y, c1.w, c.y0);
            sid[t] = vg;
        }
        __syncthreads();
        const int nb = min(BATCH, (int)(r.y - base));
        for (int sub = 0; sub < nb; sub += SUB) {
            const int ns = min(SUB, nb - sub);
            for (int jj = 0; jj < ns; ++jj) {
                const int k = sub + jj;
                float contrib = 0.f;
                if (warp_rows_hit(sR[k], warp) && !done) {
                    const float4 a = sA[k];
                    const float2 b = sB[k];
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
                W[jj * WSTRIDE + t] = contrib;
            }
            __syncthreads();
            const int j = t >> 3;
            const float s = table_sum(W, j < ns ? sR[sub + j] : make_int2(0, -1));
            if ((t & 7) == 0 && j < ns && s != 0.f) atomicAdd(&A[sid[sub + j]], s);
            __syncthreads();
        }
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
// Each pixel gathers; no reduction is needed.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_splat_fwd(const uint2 *__restrict__ rangesI, const uint32_t *__restrict__ vals, const ImgRec *__restrict__ img,
            const CompRec *__restrict__ comp, const float *__restrict__ A, const ViewDev *__restrict__ views, int V,
            float cut, const StatusDev *st, float *__restrict__ images) {
    __shared__ float4 sA[BATCH];
    __shared__ float2 sB[BATCH];
    __shared__ int2 sR[BATCH];
    const int t = threadIdx.x, warp = t >> 5;
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
            sR[t] = tile_rows(i0.y, i1.z, c.y0);
        }
        __syncthreads();
        const int nb = min(BATCH, (int)(r.y - base));
        for (int k = 0; k < nb; ++k) {
            if (!warp_rows_hit(sR[k], warp)) continue;
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
    __shared__ int2 sR[BATCH];
    __shared__ uint32_t sid[BATCH];
    __shared__ float W[SUB * WSTRIDE];
    const int t = threadIdx.x, warp = t >> 5;
    const TileCtx c = tile_ctx(views, V, blockIdx.x);
    const uint2 r = rangesI[blockIdx.x];
    const float fx = (float)c.px, fy = (float)c.py;
    const float g = c.inside ? dLdS[c.pix] : 0.f;
    if (__syncthreads_count(g != 0.f) == 0) return;
    const float colx = (float)(c.x0 + (t & 7));
    for (uint32_t base = r.x; base < r.y; base += BATCH) {
        __syncthreads();
        const uint32_t jload = base + t;
        if (jload < r.y) {
            const uint32_t vg = vals[jload];
            const float4 *ip = reinterpret_cast<const float4 *>(img + vg);
            const float4 i0 = ip[0], i1 = ip[1];
            sA[t] = i0;
            sC[t] = i1.x;
            sR[t] = tile_rows(i0.y, i1.z, c.y0);
            sid[t] = vg;
        }
        __syncthreads();
        const int nb = min(BATCH, (int)(r.y - base));
        for (int sub = 0; sub < nb; sub += SUB) {
            const int ns = min(SUB, nb - sub);
            for (int jj = 0; jj < ns; ++jj) {
                const int k = sub + jj;
                float w = 0.f;
                if (warp_rows_hit(sR[k], warp)) {
                    const float4 a = sA[k];
                    const float q = gauss_q(a.z, a.w, sC[k], fx - a.x, fy - a.y);
                    if (q >= cut) w = g * ex2_approx(q);
                }
                W[jj * WSTRIDE + t] = w;
            }
            __syncthreads();
            const int j = t >> 3;
            float m[6];
            const float4 a = sA[sub + (j < ns ? j : 0)];
            table_moments(W, j < ns ? sR[sub + j] : make_int2(0, -1), colx - a.x, (float)c.y0 - a.y, m);
            if ((t & 7) == 0 && j < ns) add_moments(accI, sid[sub + j], m);
            __syncthreads();
        }
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
// float bits of alpha and the same skipped pairs as the forward; every
// factor is > 0 because T_{i+1} >= Tfloor).  Per (view, Gaussian) the
// moments of w = dL/dalpha exp(-delta_C/2).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_intensity_bwd(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals, const CompRec *__restrict__ comp,
                const ImgRec *__restrict__ img, const float4 *__restrict__ accI, const float *__restrict__ Tstop,
                const int32_t *__restrict__ last, const ViewDev *__restrict__ views, int V, float cut,
                const StatusDev *st, float4 *__restrict__ accC) {
    if (st->code != SDGR_OK) return;
    __shared__ float4 sA[BATCH];
    __shared__ float4 sB[BATCH];
    __shared__ int2 sR[BATCH];
    __shared__ uint32_t sid[BATCH];
    __shared__ float W[SUB * WSTRIDE];
    __shared__ int smax;
    const int t = threadIdx.x, warp = t >> 5;
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
    const float colx = (float)(c.x0 + (t & 7));
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
            sR[t] = tile_rows(c0.y, c1.w, c.y0);
            sid[t] = vg;
        }
        __syncthreads();
        for (int send = nb; send > 0; send -= SUB) {
            const int sub = max(0, send - SUB);
            const int ns = send - sub;
            for (int jj = ns - 1; jj >= 0; --jj) {
                const int k = sub + jj;
                float w = 0.f;
                if (warp_rows_hit(sR[k], warp) && lo + k < mylast) {
                    const float4 a = sA[k];
                    const float4 b = sB[k];
                    const float dx = __fsub_rn(fx, a.x), dy = __fsub_rn(fy, a.y);
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
                    }
                }
                W[jj * WSTRIDE + t] = w;
            }
            __syncthreads();
            const int j = t >> 3;
            float m[6];
            const float4 a = sA[sub + (j < ns ? j : 0)];
            table_moments(W, j < ns ? sR[sub + j] : make_int2(0, -1), colx - a.x, (float)c.y0 - a.y, m);
            if ((t & 7) == 0 && j < ns) add_moments(accC, sid[sub + j], m);
            __syncthreads();
        }
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
