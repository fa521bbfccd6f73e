// k_raster.cu -- steps a7, a8, a10, a11 of the rasterizer: the per-tile loops
// over depth-sorted Gaussians on the computation plane (scattering intensity,
// Section II-A-2, eq. I_i) and the layover splat on the imaging plane
// (Section II-A-3, eq. S_{n,m}), and their adjoints (Section II-B-1/2).
//
// A CTA works on one 16x16 tile at a time.  The intensity pass, the splat
// and the intensity adjoint run four warps; warp w covers the 8x8 block with
// columns 8 (w & 1) .. +7 and rows 8 (w >> 1) .. +7, two rays (pixels) per
// lane in one column.  The splat adjoint runs eight warps, Gaussian-parallel.
// Which tiles a CTA takes follows the launch's schedule (for_tiles): one CTA
// per tile, one per item of the longest-first work list, or resident CTAs
// pulling items.  The tile's instance list is staged through shared memory in
// batches (the staging batch of each kernel, a tuning knob).
//
// Culling: when a batch is staged, each Gaussian gets the set of the tile's
// pixel blocks that its K-ellipse reaches (found from the ellipse's exact
// horizontal extent over each band of four rows): eight 8x4 blocks (the
// intensity pass takes an 8x8 block as the union of two, the splat adjoint
// walks them), or sixteen 4x4 sub-blocks (the splat; the intensity adjoint
// merges them into eight 4x8 half-blocks).  A warp, or in the splat and the
// intensity adjoint each half of it (the left and right four columns of its
// block), walks only the Gaussians whose set holds its block: per 32 staged
// Gaussians one ballot gives it its hit list, which it visits in list order
// (front to back for the intensity pass, back to front for its adjoint),
// written out as byte indices (one popc per lane): a shared load per hit
// instead of a bit scan and a mask update (-7 % and -5 % of the intensity
// pass and its adjoint when they were introduced).
//
// Exponent: in a tile, a pixel's exponent of Gaussian i is a quadratic in the
// pixel's tile-local coordinates (X, Y); the six coefficients are formed when
// the batch is staged, so a pair costs five FMAs on per-thread constants
// (Horner form, column part first: the two rays of a lane share a column, so
// a lane pays seven FMAs for two).
//
// Sums over the tile's pixels per Gaussian.  The intensity pass needs only
// sum_rays alpha T (non-negative, each term <= 1): one redux.sync per hit on
// 2^-23 fixed point, kept in a register of one lane of the warp and added to
// a 32-bit shared slot once per 32 staged Gaussians.  The intensity adjoint
// needs six signed moments and uses a two-phase transpose: in phase 1 every
// ray writes its weight for each of its hit Gaussians into a 32 x 256 shared-
// memory table; in phase 2 four threads per Gaussian read the table's entries
// of that Gaussian's half-blocks and sum them as packed pairs, then meet by
// shuffles.  Entries of half-blocks that a Gaussian does not reach are never
// read.  The splat adjoint is Gaussian-parallel over its hit blocks.
#include <type_traits>

#include "sdgr_internal.cuh"

namespace sdgr {


// Staging batch sizes (Gaussian records per CTA batch; a multiple of the CTA's
// threads -- 128, or 256 for the splat adjoint -- each thread staging whole
// records).  Larger batches mean fewer
// barriers and shorter waits for the slowest warp of a batch, smaller ones
// less shared memory (more resident CTAs) and less staging past the point
// where every ray of a tile has stopped.  The intensity adjoint's weight
// table and phase-2 mapping are built around one record per thread.
static const int kStageK3[] = {512, 256};
static const int kStageK4[] = {512, 256};
static const int kStageK5[] = {1024, 512, 256};
static const int kStageK6[] = {128};

struct TileCtx {
    int v;
    int x0, y0;  // pixel coordinates of the tile's first pixel
    float x0f, y0f;  // the same as floats (converted once per tile)
    int px, py;  // this thread's pixel
    bool inside;
    int64_t pix;
    uint32_t valid;  // pixel blocks with at least one pixel inside the image
};

__device__ __forceinline__ TileCtx tile_ctx(const ViewDev *views, int V, int tile) {
    TileCtx c;
    c.v = view_of_tile(views, V, tile);
    const ViewDev &vd = views[c.v];
    const int lt = tile - vd.tile_off;
    c.x0 = (lt % vd.tiles_x) * TILE;
    c.y0 = (lt / vd.tiles_x) * TILE;
    c.x0f = (float)c.x0;
    c.y0f = (float)c.y0;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    c.px = c.x0 + 8 * (w & 1) + (l & 7);
    c.py = c.y0 + 4 * (w >> 1) + (l >> 3);
    c.inside = c.px < vd.NA && c.py < vd.NR;
    c.pix = vd.pix_off + (int64_t)c.py * vd.NA + c.px;
    c.valid = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b)
        if (c.x0 + 8 * (b & 1) < vd.NA && c.y0 + 4 * (b >> 1) < vd.NR) c.valid |= 1u << b;
    return c;
}

// n as a float for 0 <= n < 2^23, exactly: the float with bit pattern
// 0x4B000000 | n is 2^23 + n.  A logic op and an add in place of a
// conversion instruction.
__device__ __forceinline__ float small_u2f(uint32_t n) { return __fsub_rn(__uint_as_float(0x4B000000u | n), 8388608.f); }

// Packed FP32 pairs: Blackwell's two-wide FP32 instructions (fma/add/mul
// .rn.f32x2) do two IEEE round-to-nearest operations in one issue slot, on a
// pair held in a 64-bit register (element 0 in the low half).  Each result
// equals that of the scalar instruction on each element.
struct F2 {
    uint64_t v;
};
__device__ __forceinline__ F2 pk(float lo, float hi) {
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 unpk(F2 a) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(a.v));
    return r;
}
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
__device__ __forceinline__ F2 add2(F2 a, F2 b) {
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 sub2(F2 a, F2 b) {
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 mul2(F2 a, F2 b) {
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

// Exponent coefficients in tile-local coordinates.  With the centre (u, v)
// relative to the tile origin and the pre-scaled conic (qa, qb, qc), the
// exponent qa dx^2 + qb dx dy + qc dy^2 at dx = X - u, dy = Y - v equals
// qa X^2 + qb XY + qc Y^2 + l1 X + l2 Y + c0.  Explicit round-to-nearest
// intrinsics: the intensity pass and its adjoint get the same exponent bits
// for a pair, so they agree on which pairs are inside the cutoff (the adjoint
// divides out exactly the factors the forward multiplied in).
__device__ __forceinline__ void poly_coeffs(float u, float v, float qa, float qb, float qc, float4 &P, float2 &Q) {
    const float l1 = -__fmaf_rn(2.f * qa, u, __fmul_rn(qb, v));
    const float l2 = -__fmaf_rn(2.f * qc, v, __fmul_rn(qb, u));
    const float c0 = __fmaf_rn(__fmaf_rn(qa, u, __fmul_rn(qb, v)), u, __fmul_rn(__fmul_rn(qc, v), v));
    P = make_float4(qa, qb, qc, l1);
    Q = make_float2(l2, c0);
}

// The exponent in Horner form, column part first: with
// bx = (qa X + l1) X + c0 and my = qb X + l2 (the column's part, which the
// rays of one column share), q = (qc Y + my) Y + bx -- five FMAs for one
// ray, three plus two per ray for rays of one column.  Every kernel that
// decides a pair's cutoff evaluates it in exactly this order.
struct ColQ {
    float bx, my;
};

__device__ __forceinline__ ColQ poly_col(const float4 &P, float l2, float c0, float X) {
    ColQ c;
    c.bx = __fmaf_rn(__fmaf_rn(P.x, X, P.w), X, c0);
    c.my = __fmaf_rn(P.y, X, l2);
    return c;
}

__device__ __forceinline__ float poly_row(const float4 &P, const ColQ &c, float Y) {
    return __fmaf_rn(__fmaf_rn(P.z, Y, c.my), Y, c.bx);
}

// The same from a record laid out as R = (qa, qb, l1, l2) with qc apart (the
// intensity pass's staging layout, which needs fewer registers there).
__device__ __forceinline__ ColQ poly_col_r(const float4 &R, float c0, float X) {
    ColQ c;
    c.bx = __fmaf_rn(__fmaf_rn(R.x, X, R.z), X, c0);
    c.my = __fmaf_rn(R.y, X, R.w);
    return c;
}

__device__ __forceinline__ float poly_row_q(float qc, const ColQ &c, float Y) {
    return __fmaf_rn(__fmaf_rn(qc, Y, c.my), Y, c.bx);
}

// Tile-local rows [x, y] that the K-ellipse of a Gaussian centred at row uy
// with bounding-box half-height ry can reach (empty when x > y).
__device__ __forceinline__ int2 tile_rows(float uy, float ry, float y0) {
    float lo = ceilf(uy - ry) - y0, hi = floorf(uy + ry) - y0;
    lo = fminf(fmaxf(lo, 0.f), 16.f);
    hi = fminf(fmaxf(hi, -1.f), 15.f);
    if (!(lo <= 16.f)) lo = 0.f;  // NaN centre: keep every row, the mask test decides
    if (!(hi >= -1.f)) hi = 15.f;
    return make_int2((int)lo, (int)hi);
}

// Pixel blocks of the tile that the K-ellipse reaches.  (u, v): centre
// relative to the tile origin; q = qa dx^2 + qb dx dy + qc dy^2 (negative
// definite); rows: the tile rows of the ellipse's bounding box; cutm: the
// exponent cutoff widened by 1% so that the test stays conservative under
// rounding.  For a fixed dy the in-cutoff dx form the interval
// kx dy +- hw(dy), kx = -qb / (2 qa), hw(dy)^2 = (cutm - qs dy^2) / qa,
// qs = qc - qb^2 / (4 qa).  The right end is concave in dy and peaks at the
// ellipse's right-most point dy_R = ky dx_R (ky = -qb / (2 qc), dx_R the
// bounding-box half-width), so over a band of rows it peaks at dy_R clamped
// into the band; the left end mirrors this at -dy_R.  A block is kept when
// the band's extent overlaps its eight columns.  NaN records get no block.
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint32_t block_mask(float u, float v, float qa, float qb, float qc, float cutm, int2 rows) {
    const float kx = -0.5f * __fdividef(qb, qa);
    const float ky = -0.5f * __fdividef(qb, qc);
    const float qs = fmaf(0.5f * qb, kx, qc);
    const float qt = fmaf(0.5f * qb, ky, qa);
    const float dyR = ky * sqrt_approx(fmaxf(0.f, __fdividef(cutm, qt)));
    const float iqa = __fdividef(1.f, qa);
    uint32_t m = 0;
#pragma unroll
    for (int rb = 0; rb < 4; ++rb) {
        if (rows.x > 4 * rb + 3 || rows.y < 4 * rb) continue;
        const float ya = (float)(4 * rb) - v, yb = ya + 3.f;
        const float tR = fminf(fmaxf(dyR, ya), yb), tL = fminf(fmaxf(-dyR, ya), yb);
        const float hR = sqrt_approx(fmaxf(0.f, (cutm - qs * tR * tR) * iqa));
        const float hL = sqrt_approx(fmaxf(0.f, (cutm - qs * tL * tL) * iqa));
        const float xmax = fmaf(kx, tR, hR), xmin = fmaf(kx, tL, -hL);
        const float xa = -u, xb = 8.f - u;
        if (xmax >= xa && xmin <= xa + 7.f) m |= 1u << (2 * rb);
        if (xmax >= xb && xmin <= xb + 7.f) m |= 2u << (2 * rb);
    }
    return m;
}

// The same test on the tile's sixteen 4 x 4 sub-blocks: bit 4 rb + cb for
// rows 4 rb .. 4 rb + 3 and columns 4 cb .. 4 cb + 3.
__device__ __forceinline__ uint32_t subblock_mask(float u, float v, float qa, float qb, float qc, float cutm,
                                                  int2 rows) {
    const float kx = -0.5f * __fdividef(qb, qa);
    const float ky = -0.5f * __fdividef(qb, qc);
    const float qs = fmaf(0.5f * qb, kx, qc);
    const float qt = fmaf(0.5f * qb, ky, qa);
    const float dyR = ky * sqrt_approx(fmaxf(0.f, __fdividef(cutm, qt)));
    const float iqa = __fdividef(1.f, qa);
    uint32_t m = 0;
#pragma unroll
    for (int rb = 0; rb < 4; ++rb) {
        if (rows.x > 4 * rb + 3 || rows.y < 4 * rb) continue;
        const float ya = (float)(4 * rb) - v, yb = ya + 3.f;
        const float tR = fminf(fmaxf(dyR, ya), yb), tL = fminf(fmaxf(-dyR, ya), yb);
        const float hR = sqrt_approx(fmaxf(0.f, (cutm - qs * tR * tR) * iqa));
        const float hL = sqrt_approx(fmaxf(0.f, (cutm - qs * tL * tL) * iqa));
        const float xmax = fmaf(kx, tR, hR), xmin = fmaf(kx, tL, -hL);
#pragma unroll
        for (int cb = 0; cb < 4; ++cb) {
            const float xa = (float)(4 * cb) - u;
            if (xmax >= xa && xmin <= xa + 3.f) m |= 1u << (4 * rb + cb);
        }
    }
    return m;
}

// Per-block moments of two columns at once, as pairs: W0..W3 the weights of
// rows dy .. dy + 3 of both columns, DX their column offsets; adds sum w,
// w dx, w dy, w dx^2, w dx dy, w dy^2 into the pair accumulators M (element
// i: column i's share).
__device__ __forceinline__ void block_moments2(F2 W0, F2 W1, F2 W2, F2 W3, F2 DX, F2 DY, F2 M[6]) {
    const F2 a = add2(W2, W3), b = add2(W1, a);
    const F2 sw = add2(W0, b);                 // sum w_i
    const F2 s1 = add2(add2(b, a), W3);        // sum w_i i
    const F2 t = add2(a, add2(W3, W3));        // w_2 + 3 w_3
    const F2 s2 = add2(s1, add2(t, t));        // sum w_i i^2
    const F2 py = fma2(DY, sw, s1);            // sum w_i (dy + i)
    const F2 pyy = fma2(DY, add2(py, s1), s2); // sum w_i (dy + i)^2
    const F2 px = mul2(sw, DX);
    M[0] = add2(M[0], sw);
    M[1] = add2(M[1], px);
    M[2] = add2(M[2], py);
    M[3] = fma2(px, DX, M[3]);
    M[4] = fma2(py, DX, M[4]);
    M[5] = add2(M[5], pyy);
}

// Block list of an 8-bit block set m: the indices of its set bits in
// increasing order, four bits each (the i-th in bits 4i .. 4i + 3), and 8 in
// the nibbles past them (a block of zeros for a loop that walks more blocks
// than the set has).  Built once per CTA into a 256-entry shared table, so
// that a phase-2 loop walks a Gaussian's blocks with a shift and a mask per
// block.
__device__ __forceinline__ uint32_t block_list(uint32_t m) {
    uint32_t l = 0u;
    int n = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b)
        if ((m >> b) & 1u) {
            l |= (uint32_t)b << (4 * n);
            ++n;
        }
    return n < 8 ? l | (0x88888888u << (4 * n)) : l;
}

// Hit list of this warp among the staged Gaussians [k0, k0 + n) (n <= 32).
__device__ __forceinline__ uint32_t warp_hits(const uint32_t *sM, int k0, int n) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool h = lane < n && ((sM[k0 + (lane < n ? lane : 0)] >> warp) & 1u);
    return __ballot_sync(0xffffffffu, h);
}

__device__ __forceinline__ float cut_margin(float cut) { return cut * 1.01f; }

// Phase-2 order of the staged Gaussians [k0, k0 + n) (n <= 32): ascending
// block count, so that the four Gaussians that one warp sums side by side
// have about the same number of blocks.  Called by a whole warp; writes
// perm[0..31] (slots past n hold Gaussians with no block).
__device__ __forceinline__ void order_by_blocks(const uint32_t *sM, int k0, int n, uint8_t *perm) {
    const int lane = threadIdx.x & 31;
    const int pc = lane < n ? __popc(sM[k0 + (lane < n ? lane : 0)]) : 0;
    const uint32_t lt = (1u << lane) - 1u;
    int rank = 0;
#pragma unroll
    for (int p = 0; p <= 8; ++p) {
        const uint32_t b = __ballot_sync(0xffffffffu, pc == p);
        rank += p < pc ? __popc(b) : (p == pc ? __popc(b & lt) : 0);
    }
    perm[rank] = (uint8_t)lane;
}

// Opacity of a pair from the record's opacity field o (o itself, or the
// optical depth tau of the Beer-Lambert mode AM = 1) and the profile
// e = exp(-delta/2) (0 for a pair that is skipped).  Explicit round-to-nearest
// operations, reproducible wherever a pair is evaluated.
template <int AM>
__device__ __forceinline__ float alpha_of(float o, float e) {
    if (AM == 0) return __fmul_rn(o, e);
    const float y = __fmul_rn(o, e);  // tau G
    // 1 - exp(-y): below 1/8 a series (no cancellation; truncation below
    // y^7 / 5040), above it through ex2
    float p = __fmaf_rn(y, -1.f / 720.f, 1.f / 120.f);
    p = __fmaf_rn(y, p, -1.f / 24.f);
    p = __fmaf_rn(y, p, 1.f / 6.f);
    p = __fmaf_rn(y, p, -0.5f);
    p = __fmaf_rn(y, p, 1.f);
    const float series = __fmul_rn(y, p);
    const float direct = __fsub_rn(1.f, ex2_approx(__fmul_rn(-LOG2E, y)));
    return y < 0.125f ? series : direct;
}

// Opacity folded into the exponent (alpha_mode 0): alpha = o exp2(q) =
// exp2(q + log2 o), so the staged record carries c0 + log2 o in place of c0
// and the pair's cutoff q >= cut becomes q + log2 o >= cut + log2 o.  The
// intensity pass and its adjoint stage the same record bits (the same
// instructions on the same inputs), so they take the same cutoff decisions
// and the same alpha bits.  o = 0 gives log2 o = -inf: the cutoff test
// passes and alpha = exp2(-inf) = 0.
__device__ __forceinline__ void fold_opacity(float o, float cut, float &c0, float &cutq) {
    const float lo = __log2f(o);
    c0 = __fadd_rn(c0, lo);
    cutq = __fadd_rn(cut, lo);
}

// Calls f(0), ..., f(N - 1) as straight-line code.  (A `for` loop over a
// compile-time trip count, even with `#pragma unroll`, costs the staging code
// six registers here.)
template <int N, typename F>
__device__ __forceinline__ void unrolled(F &&f) {
    if constexpr (N > 0) {
        unrolled<N - 1>(f);
        f(N - 1);
    }
}

// Runs body(tile) for the tiles this CTA owns under the launch's schedule.
template <typename F>
__device__ __forceinline__ void for_tiles(const TileSched &sc, const StatusDev *st, F &&body) {
    if (!sc.order) {
        body((int)blockIdx.x);
        return;
    }
    const int n = sc.work->count[sc.plane];
    if (sc.persistent_grid == 0) {
        if ((int)blockIdx.x < n) {
            const int tile = sc.order[blockIdx.x];
            if (SDGR_IN_BOUNDS(st, (unsigned)tile < (unsigned)sc.ntiles)) body(tile);
        }
        return;
    }
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&sc.work->next[sc.slot], 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();  // every thread has read s_item before it is overwritten
        if (item >= n) break;
        const int tile = sc.order[item];
        if (SDGR_IN_BOUNDS(st, (unsigned)tile < (unsigned)sc.ntiles)) body(tile);
    }
    (void)st;
}

// A staged list entry must be a (view, Gaussian) slot of the tile's view.
__device__ __forceinline__ bool vg_ok(const StatusDev *st, const ViewDev &vd, uint32_t vg) {
    (void)st;
    (void)vd;
    (void)vg;
    return SDGR_IN_BOUNDS(st, (uint64_t)((int64_t)vg - vd.vg_off) < (uint64_t)(uint32_t)vd.N);
}

// Stage one computation-plane record: exponent coefficients, block set and
// the Gaussian's (view, Gaussian) slot.
__device__ __forceinline__ void stage_comp(const CompRec *__restrict__ comp, uint32_t vg, const TileCtx &c, float cutm,
                                           float4 &P, float2 &Q, uint32_t &mask, float2 &uv, float2 &oP) {
    const float4 *cp = reinterpret_cast<const float4 *>(comp + vg);
    const float4 c0 = cp[0], c1 = cp[1];  // (ux, uy, qa, qb), (qc, o, P, ry)
    oP = make_float2(c1.y, c1.z);
    const float u = __fsub_rn(c0.x, c.x0f), v = __fsub_rn(c0.y, c.y0f);
    poly_coeffs(u, v, c0.z, c0.w, c1.x, P, Q);
    mask = block_mask(u, v, c0.z, c0.w, c1.x, cutm, tile_rows(c0.y, c1.w, c.y0f)) & c.valid;
    uv = make_float2(u, v);
}

// ---------------------------------------------------------------------------
// a7: intensity pass.  Per ray (cell centre): T = 1; for each Gaussian in
// depth order: alpha = o exp(-delta/2) within the cutoff; the Gaussian
// receives alpha T; T *= 1 - alpha.  The ray stops once T < Tfloor (the pair
// that takes it below the floor is the last one it takes).  For the adjoint a
// ray that stopped records the negated index just past its stopping Gaussian
// and the transmittance in front of it; any other ray its transmittance
// behind its last pair and an index past its last in-cutoff Gaussian (just
// past the last Gaussian that reaches its warp's block).  The pair update is
// branch-free: a pair outside the cutoff gets weight 0, which leaves T
// unchanged; a stopped ray carries T = 0.
//
// The ray carries Ts = 2^23 T (exact while T is normal).  With it one FMA
// gives the pair's fixed-point weight: fma(alpha, Ts, 2^23) lies in [2^23, 2^24], where
// floats are the integers, so its bit pattern is 0x4B000000 + round(2^23
// alpha T); the 32 lanes' patterns add up (mod 2^32) to 32 x 0x4B000000 =
// 0x60000000 (mod 2^32) plus the warp's sum, at most 2^28.
// ---------------------------------------------------------------------------
constexpr float S23 = 8388608.f;         // 2^23: scale of the intensity pass's transmittance
constexpr uint32_t S23_BITS = 0x4B000000u;  // bit pattern of 2^23

// TfloorS: the transmittance floor times 2^23.  Four warps per tile, each on
// an 8 x 8 block of rays with two rays per lane (rows r and r + 4 of the
// block); each ray's exponent is the same five-FMA quadratic, in the same
// tile-local coordinates and order, as the adjoint evaluates for it (the
// column part computed once for both rays).  A lane adds its
// two rays' fixed-point weights before the warp's redux: 64 patterns of
// 2^23 + k sum to 64 x 0x4B000000 = 0xC0000000 (mod 2^32) plus the warp's
// sum, at most 2^29.
template <int AM, int NB>
__device__ __forceinline__ void
intensity_fwd_tile(const int tile, const StatusDev *st, const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals,
                   const CompRec *__restrict__ comp, const ViewDev *__restrict__ views, int V, float cut, float TfloorS,
                   float *__restrict__ A, float *__restrict__ Tend, int32_t *__restrict__ last) {
    constexpr int NT = 128;
    constexpr int PER = NB / NT;  // records staged per thread
    __shared__ float4 sP[NB];  // (qa, qb, l1, l2)
    __shared__ float4 sQ[NB];  // (qc, c0 + log2 o, cut + log2 o, -); alpha_mode 1: (qc, c0, tau, -)
    __shared__ uint32_t sM[NB];
    __shared__ uint32_t sid[NB];
    __shared__ uint32_t sAcc[NB];  // sum of alpha T over the tile's 256 rays, in units of 2^-23 (< 2^31)
    __shared__ uint16_t sHL[4 * 32];  // per warp: its hit list of the current slice
    // per ray (thread t: rays t and t + 128) once it stopped: T in front of its
    // stopping pair, and -(list index of that pair + 1); written by its own thread
    __shared__ float sTe[2 * NT];
    __shared__ int32_t sLj[2 * NT];
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    uint16_t *const wl = sHL + 32 * w;
    int nh = 0;
    TileCtx c;
    c.v = view_of_tile(views, V, tile);
    const ViewDev &vd = views[c.v];
    {
        const int lt = tile - vd.tile_off;
        c.x0 = (lt % vd.tiles_x) * TILE;
        c.y0 = (lt / vd.tiles_x) * TILE;
        c.x0f = (float)c.x0;
        c.y0f = (float)c.y0;
        c.valid = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if (c.x0 + 8 * (b & 1) < vd.NA && c.y0 + 4 * (b >> 1) < vd.NR) c.valid |= 1u << b;
    }
    const int X = 8 * (w & 1) + (lane & 7), Y = 8 * (w >> 1) + (lane >> 3);
    const int px = c.x0 + X, py0 = c.y0 + Y, py1 = py0 + 4;
    const bool in0 = px < vd.NA && py0 < vd.NR, in1 = px < vd.NA && py1 < vd.NR;
    const float fX = (float)X, fY0 = (float)Y, fY1 = (float)(Y + 4);
    const F2 S23P = pk(S23, S23);
    const uint2 r = ranges[tile];
    const float cutm = cut_margin(cut);
    constexpr uint32_t WARP_BIAS = 0xC0000000u;  // 64 x bits(2^23), mod 2^32
    float T0 = in0 ? S23 : 0.f, T1 = in1 ? S23 : 0.f;  // a ray outside the image takes no pair
    sLj[t] = 0;
    sLj[t + NT] = 0;
    int32_t wb = 0;  // 1 + the list index of the warp's last hit
    // opacities of the lane's two pairs with the staged record at byte offset off
    const auto alphas = [&](uint32_t off, float &a0, float &a1) {
        const float4 P = *reinterpret_cast<const float4 *>(reinterpret_cast<const char *>(sP) + off);
        const float4 Q = *reinterpret_cast<const float4 *>(reinterpret_cast<const char *>(sQ) + off);
        const ColQ cq = poly_col_r(P, Q.y, fX);
        const float q0 = poly_row_q(Q.x, cq, fY0);
        const float q1 = poly_row_q(Q.x, cq, fY1);
        if constexpr (AM == 0) {  // Q.z: the folded cutoff; the exponent includes log2 o
            a0 = q0 >= Q.z ? ex2_approx(q0) : 0.f;
            a1 = q1 >= Q.z ? ex2_approx(q1) : 0.f;
        } else {  // Q.z: the optical depth
            a0 = alpha_of<AM>(Q.z, q0 >= cut ? ex2_approx(q0) : 0.f);
            a1 = alpha_of<AM>(Q.z, q1 >= cut ? ex2_approx(q1) : 0.f);
        }
    };
    int nb = 0;  // Gaussians staged in the current batch
    uint32_t vnext[PER];  // next batch's list entries, loaded one batch ahead
    unrolled<PER>([&](int u) { vnext[u] = r.x + t + NT * u < r.y ? vals[r.x + t + NT * u] : 0u; });
    for (uint32_t base = r.x; base < r.y; base += NB) {
        if (__syncthreads_count((T0 < TfloorS) & (T1 < TfloorS)) == (int)blockDim.x) break;
        unrolled<PER>([&](int u) {
            const int k = t + NT * u;
            // the previous batch's sums: one global atomic per (tile, Gaussian)
            if (k < nb && sAcc[k] != 0u) atomicAdd(&A[sid[k]], __uint2float_rn(sAcc[k]) * (1.f / S23));
            if (base + k < r.y) {
                const uint32_t vg = vnext[u];
                float4 P;
                float2 Q, uv, oP;
                uint32_t m = 0;
                float oz = 0.f;
                if (vg_ok(st, vd, vg)) {
                    stage_comp(comp, vg, c, cutm, P, Q, m, uv, oP);
                    oz = oP.x;
                    if constexpr (AM == 0) fold_opacity(oP.x, cut, Q.y, oz);
                }
                sP[k] = make_float4(P.x, P.y, P.w, Q.x);
                sQ[k] = make_float4(P.z, Q.y, oz, 0.f);
                const uint32_t h = m | (m >> 2);  // 8 x 8 block 2 RB + cb: 8 x 4 blocks 4 RB + cb, 4 RB + 2 + cb
                sM[k] = (h & 3u) | ((h >> 2) & 0xcu);
                sid[k] = vg;
            }
            sAcc[k] = 0u;
            if (base + NB + k < r.y) vnext[u] = vals[base + NB + k];
        });
        __syncthreads();
        nb = min(NB, (int)(r.y - base));
        for (int sub = 0; sub < nb; sub += 32) {
            // this warp's hits in list order, as byte offsets of the staged records
            {
                const uint32_t hm = warp_hits(sM, sub, min(32, nb - sub));
                __syncwarp();  // every lane has read the previous slice's list
                if ((hm >> lane) & 1u) wl[__popc(hm & ((1u << lane) - 1u))] = (uint16_t)(16 * (sub + lane));
                nh = __popc(hm);
                __syncwarp();
            }
            // the warp's 64 rays are summed in fixed point by one redux per hit;
            // lane j keeps the warp's biased sum for staged Gaussian sub + j,
            // which goes to shared memory once per 32 staged Gaussians.  The
            // loop does not test the floor: a ray that falls below it is found
            // after the slice, which is then replayed for it.
            const uint32_t myoff = 16u * (uint32_t)(sub + lane);
            const float T0s = T0, T1s = T1;
            uint32_t mine = 0u;
#pragma unroll 8
            for (int i = 0; i < nh; ++i) {
                const uint32_t off = wl[i];
                float a0, a1;
                alphas(off, a0, a1);
                // both rays' fixed-point weights in one packed FMA (the same
                // roundings as two scalar ones)
                const float2 fw = unpk(fma2(pk(a0, a1), pk(T0, T1), S23P));
                const uint32_t f = __float_as_uint(fw.x) + __float_as_uint(fw.y);
                const uint32_t ws = __reduce_add_sync(0xffffffffu, f);
                mine = off == myoff ? ws : mine;
                T0 = __fmaf_rn(-a0, T0, T0);
                T1 = __fmaf_rn(-a1, T1, T1);
            }
            // Rays that fell below the floor in this slice (once per ray at
            // most): the same arithmetic again from the slice's start finds the
            // stopping pair (T in front of it at or above the floor, behind it
            // below) and takes the weights of the pairs behind it back out of
            // the sums (integers: exactly).
            const bool x0 = (T0 < TfloorS) & (T0s >= TfloorS);
            const bool x1 = (T1 < TfloorS) & (T1s >= TfloorS);
            if (__any_sync(0xffffffffu, x0 | x1)) {
                float R0 = T0s, R1 = T1s;
                for (int i = 0; i < nh; ++i) {
                    const uint32_t off = wl[i];
                    float a0, a1;
                    alphas(off, a0, a1);
                    const float N0 = __fmaf_rn(-a0, R0, R0), N1 = __fmaf_rn(-a1, R1, R1);
                    const uint32_t g0 = x0 & (R0 < TfloorS) ? __float_as_uint(__fmaf_rn(a0, R0, S23)) - S23_BITS : 0u;
                    const uint32_t g1 = x1 & (R1 < TfloorS) ? __float_as_uint(__fmaf_rn(a1, R1, S23)) - S23_BITS : 0u;
                    const uint32_t gs = __reduce_add_sync(0xffffffffu, g0 + g1);
                    mine = off == myoff ? mine - gs : mine;
                    const int32_t k1 = (int32_t)(base + 1u + (off >> 4));  // list index + 1
                    if (x0 & (R0 >= TfloorS) & (N0 < TfloorS)) {
                        sTe[t] = R0;
                        sLj[t] = -k1;
                    }
                    if (x1 & (R1 >= TfloorS) & (N1 < TfloorS)) {
                        sTe[t + NT] = R1;
                        sLj[t + NT] = -k1;
                    }
                    R0 = N0;
                    R1 = N1;
                }
                T0 = x0 ? 0.f : T0;  // a stopped ray adds nothing further
                T1 = x1 ? 0.f : T1;
            }
            if (nh > 0) wb = (int32_t)(base + 1u + (wl[nh - 1] >> 4));
            if (mine != 0u && mine != WARP_BIAS) atomicAdd(&sAcc[sub + lane], mine - WARP_BIAS);
        }
    }
    __syncthreads();
    unrolled<PER>([&](int u) {
        const int k = t + NT * u;
        if (k < nb && sAcc[k] != 0u) atomicAdd(&A[sid[k]], __uint2float_rn(sAcc[k]) * (1.f / S23));
    });
    if (in0) {
        const int64_t pix = vd.pix_off + (int64_t)py0 * vd.NA + px;
        const int32_t lj = sLj[t];
        Tend[pix] = (lj < 0 ? sTe[t] : T0) * (1.f / S23);
        last[pix] = lj < 0 ? lj : wb;
    }
    if (in1) {
        const int64_t pix = vd.pix_off + (int64_t)py1 * vd.NA + px;
        const int32_t lj = sLj[t + NT];
        Tend[pix] = (lj < 0 ? sTe[t + NT] : T1) * (1.f / S23);
        last[pix] = lj < 0 ? lj : wb;
    }
}

template <int AM, int NB>
__global__ void __launch_bounds__(128)
k_intensity_fwd(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals, const CompRec *__restrict__ comp,
                const ViewDev *__restrict__ views, int V, float cut, float TfloorS, const StatusDev *st,
                float *__restrict__ A, float *__restrict__ Tend, int32_t *__restrict__ last, const TileSched sc) {
    if (st->code != SDGR_OK) return;
    for_tiles(sc, st, [&](int tile) {
        intensity_fwd_tile<AM, NB>(tile, st, ranges, vals, comp, views, V, cut, TfloorS, A, Tend, last);
    });
}

// Grid of a raster launch: one CTA per tile (or work item), or the persistent grid.
static unsigned raster_grid(int tiles, const TileSched &sc) {
    return sc.order && sc.persistent_grid > 0 ? (unsigned)sc.persistent_grid : (unsigned)tiles;
}

cudaError_t launch_intensity_fwd(const uint2 *ranges, const uint32_t *vals, const CompRec *comp, const ViewDev *views,
                                 int V, int tiles, float cut, float Tfloor, int alpha_mode, const StatusDev *st,
                                 float *A, float *Tend, int32_t *last, const TileSched &sched, cudaStream_t s) {
    if (tiles <= 0) return cudaSuccess;
    const unsigned grid = raster_grid(tiles, sched);
    const int v = (alpha_mode ? 2 : 0) + (sched.nb == 512 ? 1 : 0);
    const float TfloorS = Tfloor * S23;  // exact: a power-of-two scale of a normal float
    switch (v) {
        case 0: k_intensity_fwd<0, 256><<<grid, TILE_PIX / 2, 0, s>>>(ranges, vals, comp, views, V, cut, TfloorS, st, A, Tend, last, sched); break;
        case 1: k_intensity_fwd<0, 512><<<grid, TILE_PIX / 2, 0, s>>>(ranges, vals, comp, views, V, cut, TfloorS, st, A, Tend, last, sched); break;
        case 2: k_intensity_fwd<1, 256><<<grid, TILE_PIX / 2, 0, s>>>(ranges, vals, comp, views, V, cut, TfloorS, st, A, Tend, last, sched); break;
        default: k_intensity_fwd<1, 512><<<grid, TILE_PIX / 2, 0, s>>>(ranges, vals, comp, views, V, cut, TfloorS, st, A, Tend, last, sched); break;
    }
    note_launch();
    return cudaGetLastError();
}

// Stage one imaging-plane record.
// SUBBLOCKS: the 16-bit set of 4 x 4 sub-blocks (without the image-edge
// mask) in place of the 8-bit set of 8 x 4 blocks.
template <bool SUBBLOCKS = false>
__device__ __forceinline__ void stage_img(const ImgRec *__restrict__ img, uint32_t vg, const TileCtx &c, float cutm,
                                          float4 &G, float2 &uv, float &cn, uint32_t &mask) {
    const float4 *ip = reinterpret_cast<const float4 *>(img + vg);
    const float4 i0 = ip[0], i1 = ip[1];  // (ux, uy, qa, qb), (qc, cn, ry, -)
    const float u = __fsub_rn(i0.x, c.x0f), v = __fsub_rn(i0.y, c.y0f);
    G = make_float4(i0.z, i0.w, i1.x, 0.f);
    uv = make_float2(u, v);
    cn = i1.y;
    if constexpr (SUBBLOCKS)
        mask = subblock_mask(u, v, i0.z, i0.w, i1.x, cutm, tile_rows(i0.y, i1.z, c.y0f));
    else
        mask = block_mask(u, v, i0.z, i0.w, i1.x, cutm, tile_rows(i0.y, i1.z, c.y0f)) & c.valid;
}

// ---------------------------------------------------------------------------
// a8: imaging splat.  S[pixel] = sum_i c_i exp(-delta_I/2) I_i, I_i = P_i A_i.
// Each pixel gathers over its hit list; no reduction is needed.  The splat
// runs four warps per tile, each on an 8 x 8 pixel block with two pixels per
// lane (rows r and r + 4 of one column): the two pixels share the column part
// of the exponent (seven FMAs for both instead of ten), the per-hit record
// loads and list walk serve two pixels, and four warps wait at a barrier
// instead of eight (-10 % against eight warps on 8 x 4 blocks).  No pixel
// depends on another, so the two 4 x 8 halves of a warp's block (its left and
// right four columns) walk hit lists of their own, culled on the tile's 4 x 4
// sub-blocks, side by side: the shorter list is padded with a null record.
// Left and right, not top and bottom: on the imaging plane the rows run along
// the slant range, which is the depth order of the list, so within 32 staged
// Gaussians the hits of a top and a bottom half come one after the other
// rather than side by side.  Every pixel is written: with a work list
// (non-empty tiles only) the caller zeroes the images first.
// ---------------------------------------------------------------------------
template <int NB>
__device__ __forceinline__ void
splat_fwd_tile(const int tile, const StatusDev *st, const uint2 *__restrict__ rangesI, const uint32_t *__restrict__ vals,
                const ImgRec *__restrict__ img, const CompRec *__restrict__ comp, const float *__restrict__ A,
                const ViewDev *__restrict__ views, int V, float cut, bool ok, float *__restrict__ images) {
    constexpr int NT = 128;
    constexpr int PER = NB / NT;  // records staged per thread
    __shared__ float4 sP[NB + 1];  // (qa, qb, qc, l1); entry NB: the null record
    __shared__ float4 sQ[NB + 1];  // (l2, c0, c I, -)
    __shared__ uint32_t sM[NB];
    __shared__ uint16_t sHL[4 * 64];  // per warp: the hit lists of its two halves in the current slice
    const int t = threadIdx.x, w = t >> 5, l = t & 31, h = l >> 4, j = l & 15;
    uint16_t *const wl = sHL + 64 * w;  // half h walks wl[32 h ..]
    if (t == 0) {  // no pixel is inside its cutoff: exponent -inf
        sP[NB] = make_float4(0.f, 0.f, 0.f, 0.f);
        sQ[NB] = make_float4(0.f, __int_as_float(0xff800000), 0.f, 0.f);
    }
    TileCtx c;
    c.v = view_of_tile(views, V, tile);
    const ViewDev &vd = views[c.v];
    {
        const int lt = tile - vd.tile_off;
        c.x0 = (lt % vd.tiles_x) * TILE;
        c.y0 = (lt / vd.tiles_x) * TILE;
        c.x0f = (float)c.x0;
        c.y0f = (float)c.y0;
        c.valid = 0;
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if (c.x0 + 8 * (b & 1) < vd.NA && c.y0 + 4 * (b >> 1) < vd.NR) c.valid |= 1u << b;
    }
    // half h of warp w: the 4 x 8 block of columns 8 (w & 1) + 4 h .. + 3; its
    // lanes take rows r and r + 4 of one column
    const int X = 8 * (w & 1) + 4 * h + (j & 3), Y = 8 * (w >> 1) + (j >> 2);
    const int px = c.x0 + X, py0 = c.y0 + Y, py1 = py0 + 4;
    const bool in0 = px < vd.NA && py0 < vd.NR, in1 = px < vd.NA && py1 < vd.NR;
    const float fX = (float)X, fY0 = (float)Y, fY1 = (float)(Y + 4);
    // sub-block bits of the warp's left half (rows 8 (w >> 1) .. + 7, two row
    // bands); the right half's are the next ones
    const uint32_t left = 0x11u << (8 * (w >> 1) + 2 * (w & 1)), right = left << 1;
    const uint2 r = ok ? rangesI[tile] : make_uint2(0u, 0u);
    const float cutm = cut_margin(cut);
    float acc0 = 0.f, acc1 = 0.f;
    uint32_t vnext[PER];
    unrolled<PER>([&](int u) { vnext[u] = r.x + t + NT * u < r.y ? vals[r.x + t + NT * u] : 0u; });
    for (uint32_t base = r.x; base < r.y; base += NB) {
        __syncthreads();
        unrolled<PER>([&](int u) {
            const int k = t + NT * u;
            if (base + k < r.y) {
                const uint32_t vg = vnext[u];
                float4 G, P;
                float2 uv, Q;
                float cn;
                uint32_t m;
                if (vg_ok(st, vd, vg)) {
                    stage_img<true>(img, vg, c, cutm, G, uv, cn, m);
                    poly_coeffs(uv.x, uv.y, G.x, G.y, G.z, P, Q);
                    sP[k] = P;
                    sQ[k] = make_float4(Q.x, Q.y, cn * comp[vg].P * A[vg], 0.f);
                    sM[k] = m;
                } else {
                    sM[k] = 0;
                }
            }
            if (base + NB + k < r.y) vnext[u] = vals[base + NB + k];
        });
        __syncthreads();
        const int nb = min(NB, (int)(r.y - base));
        for (int k0 = 0; k0 < nb; k0 += 32) {
            // the two halves' hits in list order, as byte offsets of the staged
            // records; the shorter list is padded with the null record, so that
            // both halves walk max(n0, n1) entries in lockstep
            const uint32_t mk = l < nb - k0 ? sM[k0 + l] : 0u;
            const uint32_t hm0 = __ballot_sync(0xffffffffu, (mk & left) != 0u);
            const uint32_t hm1 = __ballot_sync(0xffffffffu, (mk & right) != 0u);
            const int n0 = __popc(hm0), n1 = __popc(hm1), nh = max(n0, n1);
            const uint32_t lt = (1u << l) - 1u;
            const uint16_t me = (uint16_t)(16 * (k0 + l));
            __syncwarp();  // every lane has read the previous slice's lists
            if ((hm0 >> l) & 1u) wl[__popc(hm0 & lt)] = me;
            if ((hm1 >> l) & 1u) wl[32 + __popc(hm1 & lt)] = me;
            if (l >= n0 && l < nh) wl[l] = (uint16_t)(16 * NB);
            if (l >= n1 && l < nh) wl[32 + l] = (uint16_t)(16 * NB);
            __syncwarp();
            const uint16_t *const hl = wl + 32 * h;
#pragma unroll 8
            for (int i = 0; i < nh; ++i) {
                const uint32_t off = hl[i];
                const float4 P0 = *reinterpret_cast<const float4 *>(reinterpret_cast<const char *>(sP) + off);
                const float4 Q0 = *reinterpret_cast<const float4 *>(reinterpret_cast<const char *>(sQ) + off);
                const ColQ cq = poly_col(P0, Q0.x, Q0.y, fX);
                const float q0 = poly_row(P0, cq, fY0);
                const float q1 = poly_row(P0, cq, fY1);
                if (q0 >= cut) acc0 = fmaf(Q0.z, ex2_approx(q0), acc0);
                if (q1 >= cut) acc1 = fmaf(Q0.z, ex2_approx(q1), acc1);
            }
        }
    }
    if (in0) images[vd.pix_off + (int64_t)py0 * vd.NA + px] = acc0;
    if (in1) images[vd.pix_off + (int64_t)py1 * vd.NA + px] = acc1;
}

template <int NB>
__global__ void __launch_bounds__(128)
k_splat_fwd(const uint2 *__restrict__ rangesI, const uint32_t *__restrict__ vals, const ImgRec *__restrict__ img,
             const CompRec *__restrict__ comp, const float *__restrict__ A, const ViewDev *__restrict__ views, int V,
             float cut, const StatusDev *st, float *__restrict__ images, const TileSched sc) {
    const bool ok = st->code == SDGR_OK;
    if (!ok && sc.order) return;
    for_tiles(sc, st,
              [&](int tile) { splat_fwd_tile<NB>(tile, st, rangesI, vals, img, comp, A, views, V, cut, ok, images); });
}

cudaError_t launch_splat_fwd(const uint2 *rangesI, const uint32_t *vals, const ImgRec *img, const CompRec *comp,
                             const float *A, const ViewDev *views, int V, int tiles, float cut, const StatusDev *st,
                             float *images, const TileSched &sched, cudaStream_t s) {
    if (tiles <= 0) return cudaSuccess;
    const unsigned grid = raster_grid(tiles, sched);
    if (sched.nb == 512)
        k_splat_fwd<512><<<grid, TILE_PIX / 2, 0, s>>>(rangesI, vals, img, comp, A, views, V, cut, st, images, sched);
    else
        k_splat_fwd<256><<<grid, TILE_PIX / 2, 0, s>>>(rangesI, vals, img, comp, A, views, V, cut, st, images, sched);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a10: adjoint of the imaging splat.  Per (view, Gaussian) the moments of
// w = dL/dS * exp(-delta_I/2); the parameter adjoint turns them into
// dL/dI = c M0, dL/du_I, dL/dconic_I and dL/dc.  No pixel depends on
// another here, so the kernel is Gaussian-parallel: two threads per
// Gaussian walk its hit blocks, each thread four columns (four rows each) per
// block; the two partial moments meet by one shuffle each, and each thread
// issues three of the six atomics.  (Against eight threads of one column each,
// the per-block and per-Gaussian work is shared by four times the pixels:
// -13 %.)  A thread's four columns form two pairs (c, c + 2) that run through
// packed FP32 pair instructions -- the exponent's steps down the columns, the
// weights and the moment sums -- two columns per issue slot (-10 %); the
// dL/dS table interleaves the two columns of a pair, so that one float4 load
// holds two rows of both.
// ---------------------------------------------------------------------------
template <int NB>
__device__ __forceinline__ void
splat_bwd_tile(const int tile, const StatusDev *st, const uint2 *__restrict__ rangesI, const uint32_t *__restrict__ vals,
               const ImgRec *__restrict__ img, const float *__restrict__ dLdS, const ViewDev *__restrict__ views, int V,
               float cut, float4 *__restrict__ accI, const uint32_t *sBL) {
    constexpr int PER = NB / 256;  // records staged per thread
    __shared__ float4 sG[NB];  // (qa, qb, qc, -)
    __shared__ float2 sU[NB];  // tile-local centre
    __shared__ uint32_t sM[NB];
    __shared__ uint32_t sid[NB];
    __shared__ uint8_t sperm[NB];
    // dL/dS of the tile's pixels, then a block of zeros (block index 8 of the
    // padded block lists).  Per 8 x 4 block 32 entries: columns c and c + 2
    // (c = 0, 1, 4, 5) interleaved as pairs, row by row, so that a float4 holds
    // two rows of two columns and its halves are the pairs of the packed loop
    __shared__ __align__(16) float sg[TILE_PIX + 32];
    const int t = threadIdx.x, warp = t >> 5;
    const TileCtx c = tile_ctx(views, V, tile);
    const uint2 r = rangesI[tile];
    const float g = c.inside ? dLdS[c.pix] : 0.f;
    {
        const int col = t & 7, row = (t >> 3) & 3;
        sg[32 * warp + 8 * (((col >> 2) << 1) | (col & 1)) + 2 * row + ((col >> 1) & 1)] = g;
    }
    if (t < 32) sg[TILE_PIX + t] = 0.f;
    if (__syncthreads_count(g != 0.f) == 0) return;
    const float cutm = cut_margin(cut);
    uint32_t vnext[PER];  // next batch's list entries, loaded one batch ahead
    unrolled<PER>([&](int u) { vnext[u] = r.x + t + 256 * u < r.y ? vals[r.x + t + 256 * u] : 0u; });
    for (uint32_t base = r.x; base < r.y; base += NB) {
        __syncthreads();
        unrolled<PER>([&](int u) {
            const int k = t + 256 * u;
            if (base + k < r.y) {
                const uint32_t vg = vnext[u];
                float4 G;
                float2 uv;
                float cn;
                uint32_t m = 0;
                if (vg_ok(st, views[c.v], vg)) stage_img(img, vg, c, cutm, G, uv, cn, m);
                sG[k] = G;
                sU[k] = uv;
                sM[k] = m;
                sid[k] = vg;
            }
            if (base + NB + k < r.y) vnext[u] = vals[base + NB + k];
        });
        __syncthreads();
        const int nb = min(NB, (int)(r.y - base));
        for (int j0 = warp * 32; j0 < nb; j0 += 256) order_by_blocks(sM, j0, min(32, nb - j0), sperm + j0);
        __syncthreads();
        // two threads per Gaussian, each four columns (c2, c2 + 2, c2 + 4,
        // c2 + 6) of every block; 128 Gaussians at a time, a warp's sixteen
        // in one 32-entry window (sorted by block count).  The two warps of a
        // window swap halves every other round, so that neither takes the
        // heavier half every time and waits at the next barrier are even.
        for (int j0 = 0; j0 < nb; j0 += 128) {
            const int g = t >> 1, c2 = t & 1;
            const int w0 = j0 + (g & 96);
            const int k = w0 < nb ? w0 + sperm[w0 + ((g & 31) ^ (((j0 >> 7) & 1) << 4))] : nb;
            const int ks = k < nb ? k : 0;
            const uint32_t mb = k < nb ? sM[k] : 0u;
            uint32_t bl = sBL[mb];
            const int cnt = __popc(mb);
            const float4 G = sG[ks];
            const F2 QC2 = pk(2.f * G.z, 2.f * G.z);
            const float gy2 = 2.f * G.y, gx4 = 4.f * G.x, qc2s = 2.f * G.z;
            const float2 uv = sU[ks];
            const float dxa0 = (float)c2 - uv.x, dy00 = -uv.y;
            F2 M[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) M[q] = pk(0.f, 0.f);
            const int rounds = __reduce_max_sync(0xffffffffu, cnt);
            for (int i = 0; i < rounds; ++i) {
                const int b = (int)(bl & 15u);  // 8 past the Gaussian's blocks: zeros
                bl >>= 4;
                const float *src = sg + 32 * b + 8 * c2;
                const float dxa = (b & 1) ? dxa0 + 8.f : dxa0;
                const float dy0 = fmaf(4.f, small_u2f((uint32_t)b >> 1), dy00);
                const F2 DY = pk(dy0, dy0);
                // columns c2 + 4 hp and c2 + 4 hp + 2 as one pair; down each
                // column the exponent by differences
#pragma unroll
                for (int hp = 0; hp < 2; ++hp) {
                    const float4 ga = *reinterpret_cast<const float4 *>(src + 16 * hp);      // rows 0, 1
                    const float4 gb = *reinterpret_cast<const float4 *>(src + 16 * hp + 4);  // rows 2, 3
                    const float dx = dxa + 4.f * (float)hp;  // the pair's first column; the second: dx + 2
                    const F2 DX = pk(dx, dx + 2.f);
                    // first column: q = qa dx^2 + qb dx dy + qc dy^2, dq its step
                    // to the next row; second column: + qa (4 dx + 4) + 2 qb dy
                    // and + 2 qb
                    const float Bq = G.y * dx;
                    const float q0 = fmaf(fmaf(G.z, dy0, Bq), dy0, G.x * dx * dx);
                    const float dq0 = fmaf(qc2s, dy0, G.z + Bq);
                    F2 q = pk(q0, q0 + fmaf(gx4, dx + 1.f, gy2 * dy0));
                    F2 dq = pk(dq0, dq0 + gy2);
                    const auto wts = [&](F2 qq, float g0, float g1) {
                        const float2 e = unpk(qq);
                        return mul2(pk(g0, g1), pk(e.x >= cut ? ex2_approx(e.x) : 0.f, e.y >= cut ? ex2_approx(e.y) : 0.f));
                    };
                    const F2 W0 = wts(q, ga.x, ga.y);
                    q = add2(q, dq);
                    dq = add2(dq, QC2);
                    const F2 W1 = wts(q, ga.z, ga.w);
                    q = add2(q, dq);
                    dq = add2(dq, QC2);
                    const F2 W2 = wts(q, gb.x, gb.y);
                    q = add2(q, dq);
                    const F2 W3 = wts(q, gb.z, gb.w);
                    block_moments2(W0, W1, W2, W3, DX, DY, M);
                }
            }
            // the thread's two columns of each pair, then the Gaussian's two
            // threads: one shuffle each; lane c2 issues the atomics of moments
            // c2, c2 + 2, c2 + 4
            float m[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const float2 h = unpk(M[q]);
                m[q] = h.x + h.y;
                m[q] += __shfl_xor_sync(0xffffffffu, m[q], 1);
            }
            if (k < nb) {
                float *dst = reinterpret_cast<float *>(accI + 2 * (size_t)sid[ks]);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float v = c2 ? m[2 * q + 1] : m[2 * q];
                    if (v != 0.f) atomicAdd(dst + 2 * q + c2, v);
                }
            }
        }
    }
}

// Four resident CTAs per SM (64 registers; the 1024-record build spills a
// few words): the packed pairs need the registers, and three CTAs per SM (no
// spills) or scalar moment sums (no spills at 64) were 4 % and 2 % slower.
template <int NB>
__global__ void __launch_bounds__(256, 4)
k_splat_bwd(const uint2 *__restrict__ rangesI, const uint32_t *__restrict__ vals, const ImgRec *__restrict__ img,
            const float *__restrict__ dLdS, const ViewDev *__restrict__ views, int V, float cut, const StatusDev *st,
            float4 *__restrict__ accI, const TileSched sc) {
    if (st->code != SDGR_OK) return;
    __shared__ uint32_t sBL[256];
    sBL[threadIdx.x] = block_list(threadIdx.x);
    __syncthreads();
    for_tiles(sc, st,
              [&](int tile) { splat_bwd_tile<NB>(tile, st, rangesI, vals, img, dLdS, views, V, cut, accI, sBL); });
}

cudaError_t launch_splat_bwd(const uint2 *rangesI, const uint32_t *vals, const ImgRec *img, const float *dLdS,
                             const ViewDev *views, int V, int tiles, float cut, const StatusDev *st, float4 *accI,
                             const TileSched &sched, cudaStream_t s) {
    if (tiles <= 0) return cudaSuccess;
    const unsigned grid = raster_grid(tiles, sched);
    if (sched.nb == 256)
        k_splat_bwd<256><<<grid, TILE_PIX, 0, s>>>(rangesI, vals, img, dLdS, views, V, cut, st, accI, sched);
    else if (sched.nb == 512)
        k_splat_bwd<512><<<grid, TILE_PIX, 0, s>>>(rangesI, vals, img, dLdS, views, V, cut, st, accI, sched);
    else
        k_splat_bwd<1024><<<grid, TILE_PIX, 0, s>>>(rangesI, vals, img, dLdS, views, V, cut, st, accI, sched);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a11: adjoint of the intensity pass.  With chat_i = dL/dI_i P_i the ray's
// share of L is sum_i chat_i alpha_i T_i, so dL/dalpha_i = T_i (chat_i - B_i),
// B_i = sum_{j>i} chat_j alpha_j prod_{i<k<j}(1 - alpha_k).  Each ray walks
// its hit list back to front from the last in-cutoff Gaussian the forward
// pass recorded: B by the suffix recursion B <- B + alpha (chat - B), T by
// undoing the forward products (T_i = T_{i+1} / (1 - alpha_i), with the same
// float bits of alpha and the same skipped pairs as the forward; every
// factor is > 0 because T_{i+1} >= Tfloor).  The pair update is branch-free
// (weight 0 outside the cutoff leaves B and T unchanged).  Per
// (view, Gaussian) the moments of w = dL/dalpha exp(-delta_C/2).
//
// Layout: four warps per tile, warp w on the 8 x 8 block of columns
// 8 (w & 1) .. and rows 8 (w >> 1) ..; its lanes hold two rays each, rows r
// and r + 4 of one column, and its two 4 x 8 halves (left: lanes 0..15,
// right: 16..31) walk hit lists of their own, culled on the tile's eight
// 4 x 8 half-blocks and padded to the same length with a staged Gaussian the
// half does not reach (weight 0: B and T stay, and the 0 written is what its
// table entry should hold).  The two rays of a lane share the column part of
// the exponent, the list entry and the record loads, and go through the
// recursion as packed FP32 pairs (the same roundings as scalar code).
//
// Phase 1 writes each ray's weight for each of its hit Gaussians into a
// 32-Gaussian x 256-pixel shared table (a lane's two rays side by side);
// phase 2 has four threads per Gaussian, thread q summing rows q and q + 4 of
// every half-block the Gaussian reaches, the six moments as packed pairs
// (the two rows), and a shuffle reduction over the four threads.
// ---------------------------------------------------------------------------
constexpr int ABATCH = 128;   // Gaussian records staged per batch: one per thread
constexpr int ASUB = 32;      // Gaussians per weight table
constexpr int AROW = 256;     // floats per weight-table row (one per pixel)

// The tile's 4 x 8 half-blocks (bit 4 R + cb: rows 8 R .. 8 R + 7, columns
// 4 cb .. 4 cb + 3) that a 4 x 4 sub-block set reaches.
__device__ __forceinline__ uint32_t halves_of_subblocks(uint32_t ms) {
    const uint32_t t = ms | (ms >> 4);
    return (t & 0xfu) | ((t >> 4) & 0xf0u);
}

template <int AM>
__device__ __forceinline__ void
intensity_bwd_tile(const int tile, const StatusDev *st, const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals,
                   const CompRec *__restrict__ comp, const ImgRec *__restrict__ img, const float4 *__restrict__ accI,
                   const float *__restrict__ Tend, const int32_t *__restrict__ last,
                   const ViewDev *__restrict__ views, int V, float cut, float4 *__restrict__ accC, const uint32_t *sBL) {
    __shared__ float4 sP[ABATCH];  // (qa, qb, l1, l2)
    __shared__ float4 sQ[ABATCH];  // (qc, c0 + log2 o, cut + log2 o, chat); alpha_mode 1: (qc, c0, tau, chat)
    __shared__ float2 sU[ABATCH];  // tile-local centre
    __shared__ uint32_t sM[ABATCH];  // half-block set
    __shared__ uint32_t sid[ABATCH];
    __shared__ uint8_t sperm[ABATCH];
    __shared__ __align__(16) float W[ASUB * AROW];
    __shared__ __align__(16) float zero32[32];  // a half-block of zeros (phase-2 rounds past a Gaussian's list)
    __shared__ __align__(4) uint16_t sHL[4 * 64];  // per warp: the hit lists of its two halves
    __shared__ int smax;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31, h = lane >> 4, j16 = lane & 15;
    uint16_t *const wl = sHL + 64 * warp;
    const uint16_t *const hl = wl + 32 * h;
    if (t < 32) zero32[t] = 0.f;
    const int v = view_of_tile(views, V, tile);
    const ViewDev &vd = views[v];
    const int lt = tile - vd.tile_off;
    const int x0 = (lt % vd.tiles_x) * TILE, y0 = (lt / vd.tiles_x) * TILE;
    const float x0f = (float)x0, y0f = (float)y0;
    uint32_t valid8 = 0;  // half-blocks with a pixel inside the image
#pragma unroll
    for (int b = 0; b < 8; ++b)
        if (x0 + 4 * (b & 3) < vd.NA && y0 + 8 * (b >> 2) < vd.NR) valid8 |= 1u << b;
    // this lane's rays: column X, rows Y and Y + 4 (tile-local)
    const int X = 8 * (warp & 1) + 4 * h + (j16 & 3), Y = 8 * (warp >> 1) + (j16 >> 2);
    const float fX = (float)X, fY0 = (float)Y, fY1 = (float)(Y + 4);
    const int hbit = 4 * (warp >> 1) + 2 * (warp & 1);  // the left half's half-block; the right: hbit + 1
    const int toff = 32 * (hbit + h) + 2 * j16;         // the lane's two table entries
    const uint2 r = ranges[tile];
    int mylast[2];
    float T[2], B[2] = {0.f, 0.f};
    bool first[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int px = x0 + X, py = y0 + Y + 4 * k;
        const bool inside = px < vd.NA && py < vd.NR;
        const int64_t pix = vd.pix_off + (int64_t)py * vd.NA + px;
        const int32_t rec = inside ? last[pix] : 0;
        mylast[k] = rec < 0 ? -rec : rec;  // negative: the ray stopped at the floor there
        // a stopped ray holds T in front of its stopping pair, which it takes
        // without a division; any other ray holds T behind its last pair
        T[k] = inside ? Tend[pix] : 0.f;  // 0 outside the image: such a ray adds nothing
        first[k] = rec < 0;
    }
    if (t == 0) smax = 0;
    __syncthreads();
    if (max(mylast[0], mylast[1]) > 0) atomicMax(&smax, max(mylast[0], mylast[1]));
    __syncthreads();
    const int hi0 = smax;
    const float cutm = cut_margin(cut);
    const F2 ONE = pk(1.f, 1.f);
    uint32_t vnext = 0u;  // next batch's list entry, loaded one batch ahead
    if (hi0 > (int)r.x && t < hi0 - max((int)r.x, hi0 - ABATCH)) vnext = vals[max((int)r.x, hi0 - ABATCH) + t];
    for (int hi = hi0; hi > (int)r.x; hi -= ABATCH) {
        const int lo = max((int)r.x, hi - ABATCH);
        const int nb = hi - lo;
        __syncthreads();
        if (t < nb) {
            const uint32_t vg = vnext;
            // a record that fails the entry check reaches no pixel: exponent
            // -inf, no half-block (it may serve as a half's padding entry)
            float4 P = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 Q = make_float2(0.f, __int_as_float(0xff800000)), uv = make_float2(0.f, 0.f);
            uint32_t m = 0;
            float chat = 0.f, oz = 0.f;
            if (vg_ok(st, vd, vg)) {
                const float4 *cp = reinterpret_cast<const float4 *>(comp + vg);
                const float4 c0 = cp[0], c1 = cp[1];  // (ux, uy, qa, qb), (qc, o, P, ry)
                const float u = __fsub_rn(c0.x, x0f), w = __fsub_rn(c0.y, y0f);
                poly_coeffs(u, w, c0.z, c0.w, c1.x, P, Q);
                m = halves_of_subblocks(
                        subblock_mask(u, w, c0.z, c0.w, c1.x, cutm, tile_rows(c0.y, c1.w, y0f))) & valid8;
                uv = make_float2(u, w);
                chat = accI[2 * (size_t)vg].x * img[vg].cn * c1.z;
                oz = c1.y;
                if constexpr (AM == 0) fold_opacity(c1.y, cut, Q.y, oz);
            }
            sP[t] = make_float4(P.x, P.y, P.w, Q.x);
            sQ[t] = make_float4(P.z, Q.y, oz, chat);
            sU[t] = uv;
            sM[t] = m;
            sid[t] = vg;
        }
        {
            const int nlo = max((int)r.x, lo - ABATCH);
            if (lo > (int)r.x && t < lo - nlo) vnext = vals[nlo + t];
        }
        __syncthreads();
        // slices of 32 from the top of the batch: slice s = [nb - 32 (s + 1), nb - 32 s)
        if (warp * ASUB < nb) {
            const int send = nb - warp * ASUB, sub = max(0, send - ASUB);
            order_by_blocks(sM, sub, send - sub, sperm + warp * ASUB);
        }
        int lim[2];  // a ray takes staged Gaussians k < lim
#pragma unroll
        for (int k = 0; k < 2; ++k) lim[k] = mylast[k] - lo;
        for (int sl = 0; sl * ASUB < nb; ++sl) {
            const int send = nb - sl * ASUB, sub = max(0, send - ASUB);
            const int ns = send - sub;
            // each half's hits back to front (descending), as byte offsets 16 k
            // of the staged records k; the shorter list padded with a record of
            // the slice that the half does not reach
            int nh;
            {
                const uint32_t mk = lane < ns ? sM[sub + lane] : 0u;
                const uint32_t h0 = __ballot_sync(0xffffffffu, (mk >> hbit) & 1u);
                const uint32_t h1 = __ballot_sync(0xffffffffu, (mk >> (hbit + 1)) & 1u);
                const int n0 = __popc(h0), n1 = __popc(h1);
                nh = max(n0, n1);
                const uint32_t live = ns >= 32 ? 0xffffffffu : (1u << ns) - 1u;
                const uint16_t me = (uint16_t)(16 * (sub + lane));
                __syncwarp();  // every lane has read the previous slice's lists
                if ((h0 >> lane) & 1u) wl[__popc(h0 >> lane) - 1] = me;
                if ((h1 >> lane) & 1u) wl[32 + __popc(h1 >> lane) - 1] = me;
                if (lane >= n0 && lane < nh) wl[lane] = (uint16_t)(16 * (sub + __ffs(~h0 & live) - 1));
                if (lane >= n1 && lane < nh) wl[32 + lane] = (uint16_t)(16 * (sub + __ffs(~h1 & live) - 1));
                __syncwarp();
            }
            // table entries of staged record k for this lane's rays: byte
            // 64 (16 k) + wb = 4 ((k - sub) AROW + toff)
            static_assert(AROW * 4 == 64 * 16, "weight table row: 64 record strides");
            const int wb = 4 * toff - 4 * AROW * sub;
            const auto rec = [&](const float4 *a, uint32_t off) {
                return *reinterpret_cast<const float4 *>(reinterpret_cast<const char *>(a) + off);
            };
            const auto hit = [&](auto fast, uint32_t off, const float4 &P, const float4 &Q) {
                constexpr bool F = decltype(fast)::value;
                const ColQ cq = poly_col_r(P, Q.y, fX);
                const float q[2] = {poly_row_q(Q.x, cq, fY0), poly_row_q(Q.x, cq, fY1)};
                float2 *const wp = reinterpret_cast<float2 *>(reinterpret_cast<char *>(W) + (int)(off * 64u) + wb);
                const float cq0 = AM == 0 ? Q.z : cut;  // the folded cutoff (alpha_mode 0)
                float wv[2];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const bool in = F ? q[k] >= cq0 : (q[k] >= cq0) & ((int)(off >> 4) < lim[k]);
                    const float e = in ? ex2_approx(q[k]) : 0.f;
                    // T in front of the pair: T behind it / (1 - alpha)
                    const auto rebuild = [&](float om) {
                        const float Td = T[k] * rcp_approx(om);
                        if constexpr (F) {
                            T[k] = Td;
                        } else {
                            T[k] = (in & !first[k]) ? Td : T[k];
                            first[k] = first[k] & !in;
                        }
                    };
                    if constexpr (AM == 0) {
                        rebuild(__fsub_rn(1.f, e));
                        const float ad = e * (Q.w - B[k]);
                        B[k] += ad;
                        wv[k] = T[k] * ad;
                    } else {
                        const float alpha = alpha_of<AM>(Q.z, e);
                        const float om = __fsub_rn(1.f, alpha);
                        rebuild(om);
                        const float d = Q.w - B[k];
                        B[k] = fmaf(alpha, d, B[k]);
                        // weight of the profile: d alpha / d G = tau (1 - alpha)
                        wv[k] = T[k] * d * (e * om);
                    }
                }
                *wp = make_float2(wv[0], wv[1]);
            };
            // the hit list walked one hit at a time (stopped rays, alpha_mode 1);
            // the next hit's list entry and records are loaded before this
            // hit's table store (which the compiler cannot move them past)
            const auto walk = [&](auto fast) {
                if (nh == 0) return;
                uint32_t off = hl[0];
                float4 P = rec(sP, off), Q = rec(sQ, off);
                for (int i = 0; i < nh; ++i) {
                    const uint32_t offn = hl[min(i + 1, nh - 1)];
                    const float4 Pn = rec(sP, offn), Qn = rec(sQ, offn);
                    hit(fast, off, P, Q);
                    off = offn;
                    P = Pn;
                    Q = Qn;
                }
            };
            // alpha_mode 0, fast path (no index bound, T always rebuilt by
            // division), as a two-stage pipeline: the part of a hit that does
            // not depend on T and B (records, exponents, alpha, 1 / (1 - alpha))
            // is done two hits ahead of the recursion (-5 % of the kernel).  e is
            // alpha itself (the exponent includes log2 o); outside the cutoff
            // alpha = 0 and rcp.approx(1) = 1 (the library's device self-check),
            // so T and B stay as they are.  The weight is dL/dalpha alpha =
            // o dL/dalpha G (the parameter adjoint divides the moments by o).
            struct Pre {
                F2 E, RC;
                float chat;
                uint32_t off;
            };
            const auto pre = [&](uint32_t off) {
                const float4 P = rec(sP, off), Q = rec(sQ, off);
                const ColQ cq = poly_col_r(P, Q.y, fX);
                const float q0 = poly_row_q(Q.x, cq, fY0), q1 = poly_row_q(Q.x, cq, fY1);
                Pre r;
                r.E = pk(q0 >= Q.z ? ex2_approx(q0) : 0.f, q1 >= Q.z ? ex2_approx(q1) : 0.f);
                const float2 om = unpk(sub2(ONE, r.E));
                r.RC = pk(rcp_approx(om.x), rcp_approx(om.y));
                r.chat = Q.w;
                r.off = off;
                return r;
            };
            const auto apply = [&](const Pre &c) {
                const F2 TT = mul2(pk(T[0], T[1]), c.RC);
                const F2 AD = mul2(c.E, pk(c.chat - B[0], c.chat - B[1]));
                const float2 b2 = unpk(add2(pk(B[0], B[1]), AD)), t2 = unpk(TT);
                T[0] = t2.x;
                T[1] = t2.y;
                B[0] = b2.x;
                B[1] = b2.y;
                *reinterpret_cast<float2 *>(reinterpret_cast<char *>(W) + (int)(c.off * 64u) + wb) = unpk(mul2(TT, AD));
            };
            // fast path: no ray of the warp is a stopped one still behind its
            // stopping pair (walking back to front) -- then the forward pass
            // took every in-cutoff pair still ahead (no index bound), and T is
            // always rebuilt by division
            if (__all_sync(0xffffffffu, !(first[0] | first[1]))) {
                if constexpr (AM == 0) {
                    if (nh > 0) {
                        Pre cur = pre(hl[0]), nxt = pre(hl[min(1, nh - 1)]);
                        for (int i = 0; i < nh; ++i) {
                            const Pre nn = pre(hl[min(i + 2, nh - 1)]);
                            apply(cur);
                            cur = nxt;
                            nxt = nn;
                        }
                    }
                } else {
                    walk(std::true_type{});
                }
            } else {
                walk(std::false_type{});
            }
            __syncthreads();
            // phase 2: four threads per Gaussian (slots sorted by half-block
            // count, so that the eight Gaussians of a warp take about as many
            // rounds); thread q sums rows q and q + 4 of both column pairs of
            // each half-block.  Per float4 (rows q, q + 4 of columns c, c + 1):
            // A, B the two columns' pairs, S = A + B; with dx the column c
            // offset, sum w dx = dx S + B, sum w dx^2 = dx^2 S + (2 dx + 1) B.
            // The first float4 read alternates with the slot, so that the two
            // Gaussians of a quarter-warp load disjoint banks.
            {
                const int slot = t >> 2, q = t & 3;
                const int jg = sperm[sl * ASUB + slot];
                const bool valid = jg < ns;
                const uint32_t mh = valid ? sM[sub + jg] & 0xffu : 0u;
                uint32_t bl = sBL[mh];
                const int cnt = __popc(mh);
                const float2 uv = sU[sub + (valid ? jg : 0)];
                const float *const wr = W + jg * AROW + 8 * q;
                const int s0 = (q + slot) & 1;
                // column offsets from the centre of the thread's column pairs
                // in half-block column band 0 (the band's 4 cb is added per
                // round), and of its rows in half-block row 0
                const F2 DXB0 = pk((float)(2 * s0) - uv.x, (float)(2 * s0) - uv.x);
                const F2 DXB1 = pk((float)(2 - 2 * s0) - uv.x, (float)(2 - 2 * s0) - uv.x);
                const F2 DYB = pk((float)q - uv.y, (float)(q + 4) - uv.y);
                const F2 TWO = pk(2.f, 2.f);
                F2 M[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) M[k] = pk(0.f, 0.f);
                const int rounds = __reduce_max_sync(0xffffffffu, cnt);
                for (int i = 0; i < rounds; ++i) {
                    const uint32_t hb = bl & 7u;
                    bl >>= 4;
                    const float *src = i < cnt ? wr + 32 * hb : zero32 + 8 * q;
                    const float ox = small_u2f(4u * (hb & 3u)), oy = small_u2f(8u * (hb >> 2));
                    const F2 DY = add2(DYB, pk(oy, oy)), DYY = mul2(DY, DY);
                    const F2 OX = pk(ox, ox);
#pragma unroll
                    for (int ss = 0; ss < 2; ++ss) {
                        const float4 v4 = *reinterpret_cast<const float4 *>(src + 4 * (s0 ^ ss));
                        const F2 DX = add2(ss ? DXB1 : DXB0, OX);
                        const F2 A = pk(v4.x, v4.y), Bc = pk(v4.z, v4.w);
                        const F2 S = add2(A, Bc);
                        const F2 P1 = fma2(DX, S, Bc);
                        M[0] = add2(M[0], S);
                        M[1] = add2(M[1], P1);
                        M[2] = fma2(DY, S, M[2]);
                        M[3] = fma2(mul2(DX, DX), S, fma2(fma2(TWO, DX, ONE), Bc, M[3]));
                        M[4] = fma2(DY, P1, M[4]);
                        M[5] = fma2(DYY, S, M[5]);
                    }
                }
                float m[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    const float2 hh = unpk(M[k]);
                    m[k] = hh.x + hh.y;
                    m[k] += __shfl_xor_sync(0xffffffffu, m[k], 1);
                    m[k] += __shfl_xor_sync(0xffffffffu, m[k], 2);
                }
                if (valid) {
                    // thread q issues moments q and, for q < 2, q + 4
                    float *dst = reinterpret_cast<float *>(accC + 2 * (size_t)sid[sub + jg]);
                    const float va = q == 0 ? m[0] : (q == 1 ? m[1] : (q == 2 ? m[2] : m[3]));
                    if (va != 0.f) atomicAdd(dst + q, va);
                    const float vb = q == 0 ? m[4] : m[5];
                    if (q < 2 && vb != 0.f) atomicAdd(dst + 4 + q, vb);
                }
            }
            __syncthreads();
        }
    }
}

template <int AM>
// Four resident CTAs per SM (106 registers): faster than five at 94
// registers (19.95-20.06 against 20.35 ms) and than three (23.0); the walk
// pipelined three hits ahead instead of two was slower (20.5).
__global__ void __launch_bounds__(128, 4)
k_intensity_bwd(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals, const CompRec *__restrict__ comp,
                const ImgRec *__restrict__ img, const float4 *__restrict__ accI, const float *__restrict__ Tend,
                const int32_t *__restrict__ last, const ViewDev *__restrict__ views, int V, float cut,
                const StatusDev *st, float4 *__restrict__ accC, const TileSched sc) {
    if (st->code != SDGR_OK) return;
    __shared__ uint32_t sBL[256];
    sBL[threadIdx.x] = block_list(threadIdx.x);
    sBL[threadIdx.x + 128] = block_list(threadIdx.x + 128);
    __syncthreads();
    for_tiles(sc, st, [&](int tile) {
        intensity_bwd_tile<AM>(tile, st, ranges, vals, comp, img, accI, Tend, last, views, V, cut, accC, sBL);
    });
}

cudaError_t launch_intensity_bwd(const uint2 *ranges, const uint32_t *vals, const CompRec *comp, const ImgRec *img,
                                 const float4 *accI, const float *Tend, const int32_t *last, const ViewDev *views,
                                 int V, int tiles, float cut, int alpha_mode, const StatusDev *st, float4 *accC,
                                 const TileSched &sched, cudaStream_t s) {
    if (tiles <= 0) return cudaSuccess;
    if (alpha_mode)
        k_intensity_bwd<1><<<raster_grid(tiles, sched), TILE_PIX / 2, 0, s>>>(ranges, vals, comp, img, accI, Tend,
                                                                              last, views, V, cut, st, accC, sched);
    else
        k_intensity_bwd<0><<<raster_grid(tiles, sched), TILE_PIX / 2, 0, s>>>(ranges, vals, comp, img, accI, Tend,
                                                                              last, views, V, cut, st, accC, sched);
    note_launch();
    return cudaGetLastError();
}

int stage_batch_options(int kernel, const int **sizes) {
    switch (kernel) {
        case 0: *sizes = kStageK3; return (int)(sizeof(kStageK3) / sizeof(int));
        case 1: *sizes = kStageK4; return (int)(sizeof(kStageK4) / sizeof(int));
        case 2: *sizes = kStageK5; return (int)(sizeof(kStageK5) / sizeof(int));
        case 3: *sizes = kStageK6; return (int)(sizeof(kStageK6) / sizeof(int));
        default: *sizes = nullptr; return 0;
    }
}

// Resident CTAs per SM of raster kernel `kernel` built for staging batch nb
// (a size stage_batch_options lists); the persistent grid is SMs times this.
int raster_blocks_per_sm(int kernel, int nb) {
    static int cache[4][3] = {};
    if (kernel < 0 || kernel > 3) return 1;
    const int vi = nb == 1024 ? 2 : (nb == 512 ? 1 : 0);
    if (cache[kernel][vi] > 0) return cache[kernel][vi];
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (kernel * 3 + vi) {
        case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_intensity_fwd<0, 256>, TILE_PIX / 2, 0); break;
        case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_intensity_fwd<0, 512>, TILE_PIX / 2, 0); break;
        case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_splat_fwd<256>, TILE_PIX / 2, 0); break;
        case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_splat_fwd<512>, TILE_PIX / 2, 0); break;
        case 6: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_splat_bwd<256>, TILE_PIX, 0); break;
        case 7: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_splat_bwd<512>, TILE_PIX, 0); break;
        case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_splat_bwd<1024>, TILE_PIX, 0); break;
        case 9: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_intensity_bwd<0>, TILE_PIX / 2, 0); break;
        default: break;
    }
    if (e != cudaSuccess || n < 1) {
        (void)cudaGetLastError();
        n = 1;
    }
    cache[kernel][vi] = n;
    return n;
}

// Device self-check of the approximate instructions whose exact values the
// kernels rely on: bit 0 -- rcp.approx of 1 is 1 (the intensity adjoint's
// fast path divides T by 1 - alpha = 1 for pairs outside the cutoff).
__global__ void k_selfcheck(uint32_t *flags) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    volatile float one = 1.f;
    uint32_t f = 0u;
    if (rcp_approx(one) == 1.f) f |= 1u;
    *flags = f;
}

cudaError_t launch_selfcheck(uint32_t *flags, cudaStream_t s) {
    k_selfcheck<<<1, 32, 0, s>>>(flags);
    note_launch();
    return cudaGetLastError();
}

// Diagnostic: in-cutoff (pixel, Gaussian) pairs of every tile of one plane.
template <typename Rec>
__global__ void __launch_bounds__(256)
k_count_pairs(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ vals, const Rec *__restrict__ rec,
              const ViewDev *__restrict__ views, int V, float cut, unsigned long long *out) {
    constexpr int CB = TILE_PIX;  // records staged per batch: one per thread of the launch
    __shared__ float4 sA[CB];
    __shared__ float sC[CB];
    const int t = threadIdx.x;
    const TileCtx c = tile_ctx(views, V, blockIdx.x);
    const uint2 r = ranges[blockIdx.x];
    const float fx = (float)c.px, fy = (float)c.py;
    unsigned int n = 0;
    for (uint32_t base = r.x; base < r.y; base += CB) {
        __syncthreads();
        const uint32_t j = base + t;
        if (j < r.y) {
            const float4 *p = reinterpret_cast<const float4 *>(rec + vals[j]);
            sA[t] = p[0];
            sC[t] = p[1].x;
        }
        __syncthreads();
        const int nb = min(CB, (int)(r.y - base));
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
