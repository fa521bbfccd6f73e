// k_preprocess.cu -- steps a1-a5 of the rasterizer: activations, 3D
// covariance, world->radar transform and the projections onto the
// computation and imaging planes (Mapping and Projection Algorithm,
// Section II-A-1 of SAR-GS, eqs. G(x), W, R_r, Sigmaprime, x_r, x_C, x_i).
//
// One thread per (view, Gaussian).  Reads the three float4 of the Gaussian
// (48 B, coalesced) and writes two 32-byte plane records, two tile
// rectangles, two instance counts and the float32 depth key.
#include "sdgr_internal.cuh"

namespace sdgr {

// ---------------------------------------------------------------------------
// Plan upload: the per-call view / scene tables travel as kernel parameters
// (no pageable-memory copy, so the upload can be captured into a graph).
// ---------------------------------------------------------------------------
constexpr int BLOB_VEC = 1000;  // 16,000 bytes of payload per launch

struct Blob {
    uint32_t n;
    uint32_t pad[3];
    uint4 data[BLOB_VEC];
};

__global__ void k_upload(const __grid_constant__ Blob b, uint4 *dst) {
    for (uint32_t i = threadIdx.x; i < b.n; i += blockDim.x) dst[i] = b.data[i];
}

cudaError_t launch_upload(const void *host_src, size_t bytes, void *dev_dst, cudaStream_t s) {
    // bytes is a multiple of 16 (tables are 16-byte aligned structs)
    const uint4 *src = static_cast<const uint4 *>(host_src);
    uint4 *dst = static_cast<uint4 *>(dev_dst);
    size_t nvec = (bytes + 15) / 16;
    Blob blob;  // host staging only; its contents are copied into each launch
    for (size_t off = 0; off < nvec; off += BLOB_VEC) {
        size_t n = nvec - off < (size_t)BLOB_VEC ? nvec - off : (size_t)BLOB_VEC;
        blob.n = (uint32_t)n;
        for (size_t k = 0; k < n; ++k) blob.data[k] = src[off + k];
        k_upload<<<1, 256, 0, s>>>(blob, dst + off);
        note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Tile rectangle of the K-ellipse of a 2D Gaussian with covariance
// (sxx, sxy, syy) centred at (ux, uy): the ellipse d^T Sigma^-1 d <= K^2 lies
// in |dx| <= K sqrt(sxx), |dy| <= K sqrt(syy).  A small margin keeps the
// float32 box a superset of the pixels the float64 reference includes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tile_rect(float ux, float uy, float sxx, float syy, float K, int NA, int NR,
                                              uint2 &rect, int4 &pix) {
    float rx = ellipse_ry(sxx, K);
    float ry = ellipse_ry(syy, K);
    float fx0 = ceilf(ux - rx), fx1 = floorf(ux + rx);
    float fy0 = ceilf(uy - ry), fy1 = floorf(uy + ry);
    bool bad = !(fx0 <= fx1) || !(fy0 <= fy1) || fx1 < 0.f || fy1 < 0.f || fx0 > (float)(NA - 1) ||
               fy0 > (float)(NR - 1);
    if (bad) {
        rect = make_uint2(0xffffffffu, 0xffffffffu);
        pix = make_int4(0, -1, 0, -1);
        return 0;
    }
    int x0 = (int)fmaxf(fx0, 0.f), x1 = (int)fminf(fx1, (float)(NA - 1));
    int y0 = (int)fmaxf(fy0, 0.f), y1 = (int)fminf(fy1, (float)(NR - 1));
    int tx0 = x0 / TILE, tx1 = x1 / TILE, ty0 = y0 / TILE, ty1 = y1 / TILE;
    rect = make_uint2((uint32_t)tx0 | ((uint32_t)tx1 << 16), (uint32_t)ty0 | ((uint32_t)ty1 << 16));
    pix = make_int4(x0, x1, y0, y1);
    return (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
}

__device__ __forceinline__ float sqrt_apx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The tiles of the rectangle that the K-ellipse reaches.  (qa, qb, qc): the
// record's exponent coefficients, q = qa dx^2 + qb dx dy + qc dy^2 (negative
// definite); cutm: the exponent cutoff widened by 1 %, as the raster kernels
// widen it for their block masks.  For a band of rows the ellipse's exact
// horizontal extent follows from the concavity of its right end in dy (it
// peaks at the ellipse's right-most point, clamped into the band; the left
// end mirrors it), the same test as the raster kernels' per-block masks, here
// per tile row over that row's pixel rows of the bounding box.  For a
// rectangle of w x h <= 32 tiles, bit r w + c is set when tile (c, r) holds a
// pixel centre of the widened ellipse, and the count is the number of bits;
// a larger rectangle keeps all its tiles (mask of all ones).  A diagonal thin
// ellipse leaves most of its rectangle empty: on the config-3 scene the exact
// sets hold 88 % of the rectangles' tiles.
__device__ __forceinline__ uint32_t tile_set(float ux, float uy, float qa, float qb, float qc, float cutm,
                                             const uint2 rect, const int4 pix, uint32_t area, uint32_t &mask) {
    mask = 0xffffffffu;
    if (area == 0u || area > 32u) return area;
    const int tx0 = (int)(rect.x & 0xffffu), tx1 = (int)(rect.x >> 16);
    const int ty0 = (int)(rect.y & 0xffffu), ty1 = (int)(rect.y >> 16);
    const int w = tx1 - tx0 + 1;
    const float kx = -0.5f * __fdividef(qb, qa);
    const float ky = -0.5f * __fdividef(qb, qc);
    const float qs = fmaf(0.5f * qb, kx, qc);
    const float qt = fmaf(0.5f * qb, ky, qa);
    const float dyR = ky * sqrt_apx(fmaxf(0.f, __fdividef(cutm, qt)));
    const float iqa = __fdividef(1.f, qa);
    uint32_t m = 0u;
    for (int ty = ty0; ty <= ty1; ++ty) {
        const int ylo = max(ty * TILE, pix.z), yhi = min(ty * TILE + TILE - 1, pix.w);
        const float ya = (float)ylo - uy, yb = (float)yhi - uy;
        const float tR = fminf(fmaxf(dyR, ya), yb), tL = fminf(fmaxf(-dyR, ya), yb);
        const float hR = sqrt_apx(fmaxf(0.f, (cutm - qs * tR * tR) * iqa));
        const float hL = sqrt_apx(fmaxf(0.f, (cutm - qs * tL * tL) * iqa));
        const float xmax = ux + fmaf(kx, tR, hR), xmin = ux + fmaf(kx, tL, -hL);
        const float c0 = fmaxf(ceilf(xmin), (float)pix.x), c1 = fminf(floorf(xmax), (float)pix.y);
        if (!(c0 <= c1)) continue;  // (NaN: no tile)
        const int t0 = (int)c0 / TILE, t1 = (int)c1 / TILE;
        const uint32_t run = (2u << (t1 - t0)) - 1u;  // t1 - t0 < w <= 32
        m |= run << ((ty - ty0) * w + (t0 - tx0));
    }
    mask = m;
    return (uint32_t)__popc(m);
}

__global__ void __launch_bounds__(256)
k_preprocess(const float4 *__restrict__ params, const float4 *__restrict__ sh, int sh_count,
             const ViewDev *__restrict__ views, int V, int64_t VG, float K,
             float eps, int norm_mode, int alpha_mode, CompRec *__restrict__ comp, ImgRec *__restrict__ img,
             BinRec *__restrict__ bin,
             uint32_t *__restrict__ dkey, uint32_t *__restrict__ dval) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < VG; i += stride) {
        const int v = view_of_vg(views, V, i);
        const ViewDev &vd = views[v];
        const int64_t g = vd.g_off + (i - vd.vg_off);
        const float4 p0 = __ldg(params + 3 * g);
        const float4 p1 = __ldg(params + 3 * g + 1);
        const float4 p2 = __ldg(params + 3 * g + 2);

        // a1: activations and rotation of the Gaussian
        const float s0 = expf(p1.x), s1 = expf(p1.y), s2 = expf(p1.z);
        const float qn = 1.0f / sqrtf(p2.x * p2.x + p2.y * p2.y + p2.z * p2.z + p2.w * p2.w);
        const float w = p2.x * qn, x = p2.y * qn, y = p2.z * qn, z = p2.w * qn;
        // the record's opacity field: o = sigmoid(logit), or the optical depth
        // tau = softplus(logit) of the Beer-Lambert opacity
        const float o = alpha_mode ? softplus(p0.w) : 1.0f / (1.0f + expf(-p0.w));
        float R[3][3];
        R[0][0] = 1.f - 2.f * (y * y + z * z); R[0][1] = 2.f * (x * y - w * z); R[0][2] = 2.f * (x * z + w * y);
        R[1][0] = 2.f * (x * y + w * z); R[1][1] = 1.f - 2.f * (x * x + z * z); R[1][2] = 2.f * (y * z - w * x);
        R[2][0] = 2.f * (x * z - w * y); R[2][1] = 2.f * (y * z + w * x); R[2][2] = 1.f - 2.f * (x * x + y * y);

        // a2: Sigma_r = (R_r R) diag(s^2) (R_r R)^T, the entries both planes use
        float M[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int k = 0; k < 3; ++k) M[a][k] = vd.r[a][0] * R[0][k] + vd.r[a][1] * R[1][k] + vd.r[a][2] * R[2][k];
        const float q0 = s0 * s0, q1 = s1 * s1, q2 = s2 * s2;
        const float S00 = M[0][0] * M[0][0] * q0 + M[0][1] * M[0][1] * q1 + M[0][2] * M[0][2] * q2;
        const float S01 = M[0][0] * M[1][0] * q0 + M[0][1] * M[1][1] * q1 + M[0][2] * M[1][2] * q2;
        const float S11 = M[1][0] * M[1][0] * q0 + M[1][1] * M[1][1] * q1 + M[1][2] * M[1][2] * q2;
        const float S02 = M[0][0] * M[2][0] * q0 + M[0][1] * M[2][1] * q1 + M[0][2] * M[2][2] * q2;
        const float S22 = M[2][0] * M[2][0] * q0 + M[2][1] * M[2][1] * q1 + M[2][2] * M[2][2] * q2;

        // a2: radar coordinates relative to the beam centre
        const float dx = p0.x - vd.c[0], dy = p0.y - vd.c[1], dz = p0.z - vd.c[2];
        const float ra = vd.r[0][0] * dx + vd.r[0][1] * dy + vd.r[0][2] * dz;  // azimuth
        const float re = vd.r[1][0] * dx + vd.r[1][1] * dy + vd.r[1][2] * dz;  // elevation
        const float rr = vd.r[2][0] * dx + vd.r[2][1] * dy + vd.r[2][2] * dz;  // slant range - R0

        // depth key: float32 rounding of the float64 slant-range offset, the
        // same operations in the same order as an IEEE double evaluation of
        // r2 . (mu - c) from left to right
        const double ddx = __dsub_rn((double)p0.x, vd.cd[0]);
        const double ddy = __dsub_rn((double)p0.y, vd.cd[1]);
        const double ddz = __dsub_rn((double)p0.z, vd.cd[2]);
        const double rho =
            __dadd_rn(__dadd_rn(__dmul_rn(vd.r2d[0], ddx), __dmul_rn(vd.r2d[1], ddy)), __dmul_rn(vd.r2d[2], ddz));
        const float key = __double2float_rn(rho) + 0.0f;  // -0 -> +0

        // a3: computation plane (x_r, y_r), cells dA x dR tan(theta)
        const float uCx = ra * vd.inv_dA + vd.offx;
        const float uCy = re * vd.inv_cy + vd.offy;
        const float cxx = S00 * vd.inv_dA * vd.inv_dA + eps;
        const float cxy = S01 * vd.inv_dA * vd.inv_cy;
        const float cyy = S11 * vd.inv_cy * vd.inv_cy + eps;
        const float idC = 1.0f / (cxx * cyy - cxy * cxy);
        // a4: imaging plane (x_r, z_r - R0), pixels dA x dR
        const float uIy = rr * vd.inv_dR + vd.offy;
        const float ixy = S02 * vd.inv_dA * vd.inv_dR;
        const float iyy = S22 * vd.inv_dR * vd.inv_dR + eps;
        const float detI = cxx * iyy - ixy * ixy;
        const float idI = 1.0f / detI;
        const float cn = norm_mode == 0 ? 0.15915494309189535f / sqrtf(detI) : 1.0f;

        CompRec cr;
        cr.ux = uCx; cr.uy = uCy;
        cr.qa = -0.5f * LOG2E * (cyy * idC);
        cr.qb = -LOG2E * (-cxy * idC);
        cr.qc = -0.5f * LOG2E * (cxx * idC);
        // view-dependent scattering: P + sum_k sh_k Y_k(direction of this view)
        float P = p1.w;
        if (sh) {
            const float4 *row = sh + 4 * g;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (4 * q >= sh_count) break;
                const float4 c4 = __ldg(row + q);
                P = fmaf(c4.x, vd.Ysh[4 * q], P);
                P = fmaf(c4.y, vd.Ysh[4 * q + 1], P);
                P = fmaf(c4.z, vd.Ysh[4 * q + 2], P);
                P = fmaf(c4.w, vd.Ysh[4 * q + 3], P);
            }
        }
        cr.o = o; cr.P = P; cr.ry = ellipse_ry(cyy, K);
        ImgRec ir;
        ir.ux = uCx; ir.uy = uIy;
        ir.qa = -0.5f * LOG2E * (iyy * idI);
        ir.qb = -LOG2E * (-ixy * idI);
        ir.qc = -0.5f * LOG2E * (cxx * idI);
        ir.cn = cn; ir.ry = ellipse_ry(iyy, K); ir.pad1 = 0.f;
        comp[i] = cr;
        img[i] = ir;

        // a5: tile rectangles of the K-ellipse on both planes, and the tiles of
        // each that the ellipse reaches
        uint2 rc, ri;
        int4 pc, pi;
        uint32_t mc, mi;
        const float cutm = -0.5f * LOG2E * K * K * 1.01f;
        uint32_t nc = tile_rect(uCx, uCy, cxx, cyy, K, vd.NA, vd.NR, rc, pc);
        uint32_t ni = tile_rect(uCx, uIy, cxx, iyy, K, vd.NA, vd.NR, ri, pi);
        nc = tile_set(uCx, uCy, cr.qa, cr.qb, cr.qc, cutm, rc, pc, nc, mc);
        ni = tile_set(uCx, uIy, ir.qa, ir.qb, ir.qc, cutm, ri, pi, ni, mi);
        if (!(o > 0.f) && !(o <= 0.f)) { nc = 0; ni = 0; }  // NaN parameters touch no tile
        BinRec b;
        b.rc = rc;
        b.ri = ri;
        b.mc = mc;
        b.mi = mi;
        b.nc = nc;
        b.ni = ni;
        bin[i] = b;
        dkey[i] = float_order_key(key);
        dval[i] = (uint32_t)i;
    }
}

cudaError_t launch_preprocess(const float4 *params, const float4 *sh, int sh_count, const ViewDev *views, int V,
                              int64_t VG, float K, float eps, int norm_mode, int alpha_mode, CompRec *comp, ImgRec *img,
                              BinRec *bin, uint32_t *dkey, uint32_t *dval, int sms, cudaStream_t s) {
    if (VG <= 0) return cudaSuccess;
    int64_t blocks = (VG + 255) / 256;
    int64_t cap = (int64_t)sms * 8;
    if (blocks > cap) blocks = cap;
    k_preprocess<<<(unsigned)blocks, 256, 0, s>>>(params, sh, sh_count, views, V, VG, K, eps, norm_mode, alpha_mode,
                                                   comp, img, bin, dkey, dval);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sdgr
