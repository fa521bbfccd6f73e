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
    // warp w covers the 8x4 pixel block (columns 8 (w & 1) .. +7, rows
    // 4 (w >> 1) .. +3); lane l sits at column l & 7, row l >> 3 of it
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    c.px = c.x0 + 8 * (w & 1) + (l & 7);
    c.py = c.y0 + 4 * (w >> 1) + (l >> 3);
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

// Tile-local columns the K-ellipse can reach, from its conic: with the
// pre-scaled conic (qa, qb, qc) and cut = -K^2 log2(e) / 2, the bounding-box
// half-width is K sqrt(Sigma_xx) = sqrt(4 cut qc / (4 qa qc - qb^2)).
__device__ __forceinline__ int2 tile_cols(float ux, float qa, float qb, float qc, float cut, int x0) {
    const float rx = sqrtf(4.f * cut * qc / (4.f * qa * qc - qb * qb)) * 1.0001f + 1e-3f;
    return tile_rows(ux, rx, x0);
}

// Bit w set when the K-ellipse's box reaches the pixel block of warp w.
__device__ __forceinline__ uint32_t warp_mask(int2 rows, int2 cols) {
    uint32_t m = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const int r0 = 4 * (w >> 1), c0 = 8 * (w & 1);
        if (rows.y >= r0 && rows.x <= r0 + 3 && cols.y >= c0 && cols.x <= c0 + 7) m |= 1u << w;
    }
    return m;
}

__device__ __forceinline__ bool warp_hit(uint32_t mask, int warp) { return (mask >> warp) & 1u; }

// Offset in the weight-table row of tile-local row r, column c (c < 8); the
// pixel in column c + 8 sits 32 entries further.
__device__ __forceinline__ int table_idx(int r, int c) { return 64 * (r >> 2) + 8 * (r & 3) + c; }

// Phase 2, one sum: every lane of the group of eight returns the sum of
// Gaussian (threadIdx.x / 8)'s table row over the rows [rows.x, rows.y].
// The four groups of a warp loop over the union of their row ranges (rows
// outside a group's range hold zeros), so every lane reads the same row at
// the same time: no divergence, no bank conflicts.
__device__ __forceinline__ int2 warp_union(int2 rows) {
    return make_int2(__reduce_min_sync(0xffffffffu, rows.x), __reduce_max_sync(0xffffffffu, rows.y));
}

__device__ __forceinline__ float table_sum(const float *W, int2 rows) {
    rows = warp_union(rows);
    const int j = threadIdx.x >> 3, c = threadIdx.x & 7;
    const float *w = W + j * WSTRIDE + c;  // thread index of pixel (row r, column c) = table_idx(r, c)
    float s = 0.f;
    for (int r = rows.x; r <= rows.y; ++r) {
        const int i = table_idx(r, 0);
        s += w[i] + w[i + 32];
    }
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    return s;
}

// Phase 2, six moments of the weights w over the pixels: sum w, w dx, w dy,
// w dx^2, w dx dy, w dy^2 with (dx, dy) = pixel - centre.  dx0 = offset of
// the thread's first column (x0 + c - ux), dy0 = y0 - uy.
__device__ __forceinline__ void table_moments(const float *W, int2 rows, float dx0, float dy0, float m[6]) {
    rows = warp_union(rows);
    const int j = threadIdx.x >> 3, c = threadIdx.x & 7;
    const float *w = W + j * WSTRIDE + c;
    const float dx1 = dx0 + 8.f;
    float m0 = 0.f, mx = 0.f, my = 0.f, mxx = 0.f, mxy = 0.f, myy = 0.f;
    for (int r = rows.x; r <= rows.y; ++r) {
        const float dy = dy0 + (float)r;
        const int i = table_idx(r, 0);
        const float w0 = w[i], w1 = w[i + 32];
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
    __shared__ uint32_t sM[BATCH];
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
            const int2 rows = tile_rows(c0.y, c1.w, c.y0);
            sR[t] = rows;
            sM[t] = warp_mask(rows, tile_cols(c0.x, c0.z, c0.w, c1.x, cut, c.x0));
            sid[t] = vg;
        }
        __syncthreads();
        const int nb = min(BATCH, (int)(r.y - base));
        for (int sub = 0; sub < nb; sub += SUB) {
            const int ns = min(SUB, nb - sub);
#pragma unroll 4
            for (int jj = 0; jj < ns; ++jj) {
                const int k = sub + jj;
                float contrib = 0.f;
                if (warp_hit(sM[k], warp) && !done) {
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
            const float s = table_sum(W, j < ns ? sR[sub + j] : make_int2(16, -1));
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
    __shared__ uint32_t sM[BATCH];
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
            sM[t] = warp_mask(tile_rows(i0.y, i1.z, c.y0), tile_cols(i0.x, i0.z, i0.w, i1.x, cut, c.x0));
        }
        __syncthreads();
        const int nb = min(BATCH, (int)(r.y - base));
        for (int k = 0; k < nb; ++k) {
            if (!warp_hit(sM[k], warp)) continue;
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
// dL/dI = c M0, dL/du_I, dL/dconic_I and dL/dc.  No pixel depends on
// another here, so the kernel is Gaussian-parallel: eight threads per
// Gaussian, each taking two columns (c, c + 8) of the rows its K-ellipse can
// reach; along a column the exponent is a quadratic in dy evaluated with two
// FMAs; dL/dS comes from shared memory; three shuffles combine the eight
// partial moments.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_splat_bwd(const uint2 *__restrict__ rangesI, const uint32_t *__restrict__ vals, const ImgRec *__restrict__ img,
            const float *__restrict__ dLdS, const ViewDev *__restrict__ views, int V, float cut, const StatusDev *st,
            float4 *__restrict__ accI) {
    if (st->code != SDGR_OK) return;
    __shared__ float4 sA[BATCH];
    __shared__ float sC[BATCH];
    __shared__ int4 sRC[BATCH];  // tile-local rows (x, y) and columns (z, w) the ellipse can reach
    __shared__ uint32_t sid[BATCH];
    __shared__ float sg[TILE_PIX];  // dL/dS of the tile's pixels, by thread index
    const int t = threadIdx.x;
    const TileCtx c = tile_ctx(views, V, blockIdx.x);
    const uint2 r = rangesI[blockIdx.x];
    const float g = c.inside ? dLdS[c.pix] : 0.f;
    sg[t] = g;
    if (__syncthreads_count(g != 0.f) == 0) return;
    const int col = t & 7;
    const float colx = (float)(c.x0 + col);
    for (uint32_t base = r.x; base < r.y; base += BATCH) {
        __syncthreads();
        const uint32_t jload = base + t;
        if (jload < r.y) {
            const uint32_t vg = vals[jload];
            const float4 *ip = reinterpret_cast<const float4 *>(img + vg);
            const float4 i0 = ip[0], i1 = ip[1];
            sA[t] = i0;
            sC[t] = i1.x;
            const int2 rows = tile_rows(i0.y, i1.z, c.y0);
            const int2 cols = tile_cols(i0.x, i0.z, i0.w, i1.x, cut, c.x0);
            sRC[t] = make_int4(rows.x, rows.y, cols.x, cols.y);
            sid[t] = vg;
        }
        __syncthreads();
        const int nb = min(BATCH, (int)(r.y - base));
        for (int j0 = 0; j0 < nb; j0 += 32) {
            const int k = j0 + (t >> 3);
            float m0 = 0.f, mx = 0.f, my = 0.f, mxx = 0.f, mxy = 0.f, myy = 0.f;
            if (k < nb) {
                const float4 a = sA[k];
                const float qc = sC[k];
                const int4 rc = sRC[k];
                const float dxa = colx - a.x, dxb = dxa + 8.f;
                // exponent along a column: qa dx^2 + (qb dx) dy + qc dy^2
                const float Aa = a.z * dxa * dxa, Ba = a.w * dxa;
                const float Ab = a.z * dxb * dxb, Bb = a.w * dxb;
                const bool va = col >= rc.z && col <= rc.w, vb = col + 8 >= rc.z && col + 8 <= rc.w;
                const float dy0 = (float)c.y0 - a.y;
                for (int rr = rc.x; rr <= rc.y; ++rr) {
                    const float dy = dy0 + (float)rr;
                    const int i = table_idx(rr, col);
                    const float qa_ = fmaf(dy, fmaf(qc, dy, Ba), Aa);
                    const float qb_ = fmaf(dy, fmaf(qc, dy, Bb), Ab);
                    const float wa = (va && qa_ >= cut) ? sg[i] * ex2_approx(qa_) : 0.f;
                    const float wb = (vb && qb_ >= cut) ? sg[i + 32] * ex2_approx(qb_) : 0.f;
                    const float xa = wa * dxa, xb = wb * dxb;
                    const float ws = wa + wb, xs = xa + xb;
                    m0 += ws;
                    mx += xs;
                    my = fmaf(ws, dy, my);
                    mxx = fmaf(xa, dxa, fmaf(xb, dxb, mxx));
                    mxy = fmaf(xs, dy, mxy);
                    myy = fmaf(ws * dy, dy, myy);
                }
            }
            float m[6] = {m0, mx, my, mxx, mxy, myy};
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                m[q] += __shfl_xor_sync(0xffffffffu, m[q], 1);
                m[q] += __shfl_xor_sync(0xffffffffu, m[q], 2);
                m[q] += __shfl_xor_sync(0xffffffffu, m[q], 4);
            }
            if (col == 0 && k < nb) add_moments(accI, sid[k], m);
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
    __shared__ uint32_t sM[BATCH];
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
            const int2 rows = tile_rows(c0.y, c1.w, c.y0);
            sR[t] = rows;
            sM[t] = warp_mask(rows, tile_cols(c0.x, c0.z, c0.w, c1.x, cut, c.x0));
            sid[t] = vg;
        }
        __syncthreads();
        for (int send = nb; send > 0; send -= SUB) {
            const int sub = max(0, send - SUB);
            const int ns = send - sub;
#pragma unroll 4
            for (int jj = ns - 1; jj >= 0; --jj) {
                const int k = sub + jj;
                float w = 0.f;
                if (warp_hit(sM[k], warp) && lo + k < mylast) {
                    const float4 a = sA[k];
                    const float4 b = sB[k];
                    const float dx = __fsub_rn(fx, a.x), dy = __fsub_rn(fy, a.y);
                    const float q = gauss_q(a.z, a.w, b.x, dx, dy);
                    if (q >= cut) {
                        const float e = ex2_approx(q);
                        const float alpha = __fmul_rn(b.y, e);
                        // relative error of a few ulp per step; the forward's rounding
                        // of 1 - alpha is undone exactly because both sides share it
                        if (!first) T = __fdividef(T, __fsub_rn(1.f, alpha));
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
            table_moments(W, j < ns ? sR[sub + j] : make_int2(16, -1), colx - a.x, (float)c.y0 - a.y, m);
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
