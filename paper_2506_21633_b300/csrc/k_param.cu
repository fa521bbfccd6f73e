// k_param.cu -- step a12 (adjoint of the projections, Section II-B-3 of
// SAR-GS: conic -> 2D covariance -> Sigma_r -> Sigma -> scale / rotation;
// pixel centres -> radar coordinates -> mean), step a13 (Adam) and step a9
// (L1 loss).  All three are HBM-bound elementwise passes.
#include "sdgr_internal.cuh"

namespace sdgr {

// dL/dq for R = R(q/|q|), from dL/dR (G) and the unit quaternion (w,x,y,z).
__device__ __forceinline__ float4 quat_grad(float w, float x, float y, float z, float qn, const float G[3][3]) {
    const float gw = 2.f * (-z * G[0][1] + y * G[0][2] + z * G[1][0] - x * G[1][2] - y * G[2][0] + x * G[2][1]);
    const float gx = 2.f * (y * G[0][1] + z * G[0][2] + y * G[1][0] - 2.f * x * G[1][1] - w * G[1][2] +
                            z * G[2][0] + w * G[2][1] - 2.f * x * G[2][2]);
    const float gy = 2.f * (-2.f * y * G[0][0] + x * G[0][1] + w * G[0][2] + x * G[1][0] + z * G[1][2] -
                            w * G[2][0] + z * G[2][1] - 2.f * y * G[2][2]);
    const float gz = 2.f * (-2.f * z * G[0][0] - w * G[0][1] + x * G[0][2] + w * G[1][0] - 2.f * z * G[1][1] +
                            y * G[1][2] + x * G[2][0] + y * G[2][1]);
    const float dot = w * gw + x * gx + y * gy + z * gz;
    return make_float4((gw - w * dot) * qn, (gx - x * dot) * qn, (gy - y * dot) * qn, (gz - z * dot) * qn);
}

// -C G C for symmetric 2x2 C = (a, b, c) and G = (p, r, s) (general-matrix
// gradient whose off-diagonal entries are both r).
__device__ __forceinline__ void neg_cgc(float a, float b, float c, float p, float r, float s, float &o00, float &o01,
                                        float &o11) {
    o00 = -(a * a * p + 2.f * a * b * r + b * b * s);
    o01 = -(a * b * p + (a * c + b * b) * r + b * c * s);
    o11 = -(b * b * p + 2.f * b * c * r + c * c * s);
}

__global__ void __launch_bounds__(256)
k_param_bwd(const float4 *__restrict__ params, const ViewDev *__restrict__ views, const SceneDev *__restrict__ scenes,
            const int32_t *__restrict__ scene_views, int n_scenes, int64_t n_gauss, float eps, int norm_mode,
            int alpha_mode, const float *__restrict__ A, const CompRec *__restrict__ comp, const float4 *__restrict__ accI,
            const float4 *__restrict__ accC, const StatusDev *st, float4 *__restrict__ grads,
            float4 *__restrict__ dsh, float *__restrict__ dens_accum, float *__restrict__ dens_count) {
    if (st->code != SDGR_OK) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_gauss; g += stride) {
        const int s = upper_index(n_scenes, g, [&](int k) { return scenes[k].g_off; });
        const SceneDev sc = scenes[s];
        const float4 p0 = __ldg(params + 3 * g), p1 = __ldg(params + 3 * g + 1), p2 = __ldg(params + 3 * g + 2);
        const float sx = expf(p1.x), sy = expf(p1.y), sz = expf(p1.z);
        const float qn = 1.0f / sqrtf(p2.x * p2.x + p2.y * p2.y + p2.z * p2.z + p2.w * p2.w);
        const float w = p2.x * qn, x = p2.y * qn, y = p2.z * qn, z = p2.w * qn;
        const float osig = 1.0f / (1.0f + expf(-p0.w));
        // factor of the computation-plane geometry: d alpha / d G is o (default;
        // the intensity adjoint's moments carry it: they are of dL/dalpha
        // alpha = o dL/dalpha G) or tau (1 - alpha) with the (1 - alpha)
        // already inside the moments
        const float o = alpha_mode ? softplus(p0.w) : 1.f;
        // dL/do from the moments of dL/dalpha alpha (default: divided by o;
        // o = 0 leaves alpha = 0 and d o / d logit = 0) or dL/dtau
        const float go_scale = alpha_mode ? 1.f : (osig > 0.f ? 1.f / osig : 0.f);
        // d o / d logit = o (1 - o); d tau / d logit = sigmoid(logit)
        const float dlogit = alpha_mode ? osig : osig * (1.f - osig);
        float R[3][3];
        R[0][0] = 1.f - 2.f * (y * y + z * z); R[0][1] = 2.f * (x * y - w * z); R[0][2] = 2.f * (x * z + w * y);
        R[1][0] = 2.f * (x * y + w * z); R[1][1] = 1.f - 2.f * (x * x + z * z); R[1][2] = 2.f * (y * z - w * x);
        R[2][0] = 2.f * (x * z - w * y); R[2][1] = 2.f * (y * z + w * x); R[2][2] = 1.f - 2.f * (x * x + y * y);
        const float ss[3] = {sx * sx, sy * sy, sz * sz};

        float dS[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};  // dL/dSigma
        float dmu[3] = {0.f, 0.f, 0.f};
        float go = 0.f, gP = 0.f;
        float dacc = 0.f, dcnt = 0.f;  // densification statistics of this call
        float gsh[15];
#pragma unroll
        for (int k = 0; k < 15; ++k) gsh[k] = 0.f;
        for (int kv = 0; kv < sc.vcount; ++kv) {
            const ViewDev &vd = views[scene_views[sc.vstart + kv]];
            const int64_t vg = vd.vg_off + (g - vd.g_off);
            // projections of this view (same formulas as the forward)
            float M[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    M[a][k] = vd.r[a][0] * R[0][k] + vd.r[a][1] * R[1][k] + vd.r[a][2] * R[2][k];
            const float S00 = M[0][0] * M[0][0] * ss[0] + M[0][1] * M[0][1] * ss[1] + M[0][2] * M[0][2] * ss[2];
            const float S01 = M[0][0] * M[1][0] * ss[0] + M[0][1] * M[1][1] * ss[1] + M[0][2] * M[1][2] * ss[2];
            const float S11 = M[1][0] * M[1][0] * ss[0] + M[1][1] * M[1][1] * ss[1] + M[1][2] * M[1][2] * ss[2];
            const float S02 = M[0][0] * M[2][0] * ss[0] + M[0][1] * M[2][1] * ss[1] + M[0][2] * M[2][2] * ss[2];
            const float S22 = M[2][0] * M[2][0] * ss[0] + M[2][1] * M[2][1] * ss[1] + M[2][2] * M[2][2] * ss[2];
            const float iA = vd.inv_dA, iC = vd.inv_cy, iR = vd.inv_dR;
            const float cxx = S00 * iA * iA + eps, cxy = S01 * iA * iC, cyy = S11 * iC * iC + eps;
            const float idC = 1.0f / (cxx * cyy - cxy * cxy);
            const float Ca = cyy * idC, Cb = -cxy * idC, Cc = cxx * idC;  // computation-plane conic
            const float ixy = S02 * iA * iR, iyy = S22 * iR * iR + eps;
            const float detI = cxx * iyy - ixy * ixy;
            const float idI = 1.0f / detI;
            const float Ia = iyy * idI, Ib = -ixy * idI, Ic = cxx * idI;  // imaging-plane conic
            const float cn = norm_mode == 0 ? 0.15915494309189535f / sqrtf(detI) : 1.0f;

            const float4 m0 = accI[2 * vg], m1 = accI[2 * vg + 1];
            const float4 n0 = accC[2 * vg], n1 = accC[2 * vg + 1];
            const float Av = A[vg];
            const float Ival = comp[vg].P * Av;  // P of this view (includes the SH term)
            // imaging plane: moments of dL/dS exp(-delta/2)
            const float dLdI = cn * m0.x;
            const float cI = Ival * cn;
            const float guIx = cI * (Ia * m0.y + Ib * m0.z);
            const float guIy = cI * (Ib * m0.y + Ic * m0.z);
            float dI00, dI01, dI11;
            neg_cgc(Ia, Ib, Ic, -0.5f * cI * m0.w, -0.5f * cI * m1.x, -0.5f * cI * m1.y, dI00, dI01, dI11);
            if (norm_mode == 0) {
                const float gc = Ival * m0.x;  // dL/dc
                dI00 += gc * (-0.5f * cn * Ia);
                dI01 += gc * (-0.5f * cn * Ib);
                dI11 += gc * (-0.5f * cn * Ic);
            }
            // computation plane: moments of dL/dalpha exp(-delta/2)
            const float guCx = o * (Ca * n0.y + Cb * n0.z);
            const float guCy = o * (Cb * n0.y + Cc * n0.z);
            float dC00, dC01, dC11;
            neg_cgc(Ca, Cb, Cc, -0.5f * o * n0.w, -0.5f * o * n1.x, -0.5f * o * n1.y, dC00, dC01, dC11);
            if (m0.x != 0.f || m0.y != 0.f || m0.z != 0.f) {  // the Gaussian received image-plane weight
                dacc += sqrtf(guIx * guIx + guIy * guIy);
                dcnt += 1.f;
            }
            go += n0.x * go_scale;
            const float dLdP = dLdI * Av;  // dL/dP of this view (P depends on the view through SH)
            gP += dLdP;
            if (dsh) {
#pragma unroll
                for (int k = 0; k < 15; ++k) gsh[k] = fmaf(dLdP, vd.Ysh[k], gsh[k]);
            }
            // Sigma' = J Sigma_r J^T + eps I  ->  dL/dSigma_r (symmetric)
            float Gr[3][3];
            Gr[0][0] = iA * iA * (dC00 + dI00);
            Gr[0][1] = Gr[1][0] = iA * iC * dC01;
            Gr[1][1] = iC * iC * dC11;
            Gr[0][2] = Gr[2][0] = iA * iR * dI01;
            Gr[2][2] = iR * iR * dI11;
            Gr[1][2] = Gr[2][1] = 0.f;
            // Sigma_r = R_r Sigma R_r^T  ->  dL/dSigma += R_r^T Gr R_r
            float Tm[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int j = 0; j < 3; ++j) Tm[a][j] = Gr[a][0] * vd.r[0][j] + Gr[a][1] * vd.r[1][j] + Gr[a][2] * vd.r[2][j];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) dS[i][j] += vd.r[0][i] * Tm[0][j] + vd.r[1][i] * Tm[1][j] + vd.r[2][i] * Tm[2][j];
            // pixel centres -> mean
            const float ga = iA * (guCx + guIx), ge = iC * guCy, gr = iR * guIy;
#pragma unroll
            for (int i = 0; i < 3; ++i) dmu[i] += vd.r[0][i] * ga + vd.r[1][i] * ge + vd.r[2][i] * gr;
        }
        // Sigma = M M^T, M = R diag(s):  dL/dM = 2 dL/dSigma M (dL/dSigma symmetric)
        const float sv[3] = {sx, sy, sz};
        float dR[3][3], ds[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const float dM = 2.f * (dS[a][0] * R[0][b] + dS[a][1] * R[1][b] + dS[a][2] * R[2][b]) * sv[b];
                ds[b] += dM * R[a][b];
                dR[a][b] = dM * sv[b];
            }
        const float4 dq = quat_grad(w, x, y, z, qn, dR);
        // accumulate (the caller zeroed grads unless it asked to accumulate)
        float4 a0 = grads[3 * g], a1 = grads[3 * g + 1], a2 = grads[3 * g + 2];
        a0.x += dmu[0]; a0.y += dmu[1]; a0.z += dmu[2]; a0.w += go * dlogit;
        a1.x += ds[0] * sx; a1.y += ds[1] * sy; a1.z += ds[2] * sz; a1.w += gP;
        a2.x += dq.x; a2.y += dq.y; a2.z += dq.z; a2.w += dq.w;
        grads[3 * g] = a0;
        grads[3 * g + 1] = a1;
        grads[3 * g + 2] = a2;
        if (dens_accum) {
            dens_accum[g] += dacc;
            dens_count[g] += dcnt;
        }
        if (dsh) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float4 d4 = dsh[4 * g + q];
                d4.x += gsh[4 * q];
                d4.y += gsh[4 * q + 1];
                d4.z += gsh[4 * q + 2];
                if (4 * q + 3 < 15) d4.w += gsh[4 * q + 3];
                dsh[4 * g + q] = d4;
            }
        }
    }
}

cudaError_t launch_param_bwd(const float4 *params, const ViewDev *views, const SceneDev *scenes,
                             const int32_t *scene_views, int n_scenes, int64_t n_gauss, float eps, int norm_mode,
                             int alpha_mode, const float *A, const CompRec *comp, const float4 *accI, const float4 *accC,
                             const StatusDev *st, float4 *grads, float4 *dsh, float *dens_accum,
                             float *dens_count, int sms, cudaStream_t s) {
    if (n_gauss <= 0) return cudaSuccess;
    int64_t blocks = (n_gauss + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    k_param_bwd<<<(unsigned)blocks, 256, 0, s>>>(params, views, scenes, scene_views, n_scenes, n_gauss, eps, norm_mode,
                                                  alpha_mode, A, comp, accI, accC, st, grads, dsh, dens_accum, dens_count);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a13: Adam, arranged like torch.optim.Adam: m <- m + (1-b1)(g - m),
// v <- b2 v + (1-b2) g^2, p <- p - (lr/bc1) m / (sqrt(v)/sqrt(bc2) + eps).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_adam(float4 *__restrict__ p, const float4 *__restrict__ g, float4 *__restrict__ m, float4 *__restrict__ v,
       int64_t n4, float4 lr0, float4 lr1, float4 lr2, float b1, float b2, float eps, float inv_bc1,
       float inv_sqrt_bc2) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const int slot = (int)(i % 3);
        const float4 lr = slot == 0 ? lr0 : (slot == 1 ? lr1 : lr2);
        float4 pp = p[i], gg = g[i], mm = m[i], vv = v[i];
        float *P = &pp.x, *G = &gg.x, *Mv = &mm.x, *Vv = &vv.x;
        const float *L = &lr.x;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            Mv[k] = Mv[k] + (1.f - b1) * (G[k] - Mv[k]);
            Vv[k] = b2 * Vv[k] + (1.f - b2) * G[k] * G[k];
            const float denom = sqrtf(Vv[k]) * inv_sqrt_bc2 + eps;
            P[k] = P[k] - (L[k] * inv_bc1) * Mv[k] / denom;
        }
        p[i] = pp;
        m[i] = mm;
        v[i] = vv;
    }
}

cudaError_t launch_adam(float4 *p, const float4 *g, float4 *m, float4 *v, int64_t n4, const float *lr, float b1,
                        float b2, float eps, int step, int sms, cudaStream_t s) {
    if (n4 <= 0) return cudaSuccess;
    const double bc1 = 1.0 - pow((double)b1, (double)step);
    const double bc2 = 1.0 - pow((double)b2, (double)step);
    int64_t blocks = (n4 + 255) / 256;
    if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
    const float4 l0 = make_float4(lr[0], lr[0], lr[0], lr[3]);
    const float4 l1 = make_float4(lr[1], lr[1], lr[1], lr[4]);
    const float4 l2 = make_float4(lr[2], lr[2], lr[2], lr[2]);
    k_adam<<<(unsigned)blocks, 256, 0, s>>>(p, g, m, v, n4, l0, l1, l2, b1, b2, eps, (float)(1.0 / bc1),
                                            (float)(1.0 / sqrt(bc2)));
    note_launch();
    return cudaGetLastError();
}

// Device-step variant: one thread advances the step counter, then the update
// reads it (two launches keep the order on the stream).
__global__ void k_step_inc(int32_t *step) { *step += 1; }

__global__ void __launch_bounds__(256)
k_adam_dev(float4 *__restrict__ p, const float4 *__restrict__ g, float4 *__restrict__ m, float4 *__restrict__ v,
           int64_t n4, float4 lr0, float4 lr1, float4 lr2, float b1, float b2, float eps, const int32_t *step) {
    const float t = (float)*step;
    const float inv_bc1 = 1.0f / (1.0f - powf(b1, t));
    const float inv_sqrt_bc2 = rsqrtf(1.0f - powf(b2, t));
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const int slot = (int)(i % 3);
        const float4 lr = slot == 0 ? lr0 : (slot == 1 ? lr1 : lr2);
        float4 pp = p[i], gg = g[i], mm = m[i], vv = v[i];
        float *P = &pp.x, *G = &gg.x, *Mv = &mm.x, *Vv = &vv.x;
        const float *L = &lr.x;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            Mv[k] = Mv[k] + (1.f - b1) * (G[k] - Mv[k]);
            Vv[k] = b2 * Vv[k] + (1.f - b2) * G[k] * G[k];
            const float denom = sqrtf(Vv[k]) * inv_sqrt_bc2 + eps;
            P[k] = P[k] - (L[k] * inv_bc1) * Mv[k] / denom;
        }
        p[i] = pp;
        m[i] = mm;
        v[i] = vv;
    }
}

cudaError_t launch_adam_dev(float4 *p, const float4 *g, float4 *m, float4 *v, int64_t n4, const float *lr, float b1,
                            float b2, float eps, int32_t *step, int sms, cudaStream_t s) {
    k_step_inc<<<1, 1, 0, s>>>(step);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || n4 <= 0) return e;
    int64_t blocks = (n4 + 255) / 256;
    if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
    const float4 l0 = make_float4(lr[0], lr[0], lr[0], lr[3]);
    const float4 l1 = make_float4(lr[1], lr[1], lr[1], lr[4]);
    const float4 l2 = make_float4(lr[2], lr[2], lr[2], lr[2]);
    k_adam_dev<<<(unsigned)blocks, 256, 0, s>>>(p, g, m, v, n4, l0, l1, l2, b1, b2, eps, step);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a9: L1 loss (mean) and its gradient.
// ---------------------------------------------------------------------------
__global__ void k_zero1(float *x) { *x = 0.f; }

__global__ void __launch_bounds__(256)
k_l1(const float *__restrict__ S, const float *__restrict__ T, int64_t n, float inv_n, float *__restrict__ dLdS,
     float *loss) {
    float acc = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float r = S[i] - T[i];
        acc += fabsf(r);
        dLdS[i] = r > 0.f ? inv_n : (r < 0.f ? -inv_n : 0.f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float wsum[8];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = 0.f;
        for (int k = 0; k < 8; ++k) b += wsum[k];
        atomicAdd(loss, b * inv_n);
    }
}

cudaError_t launch_l1(const float *S, const float *T, int64_t npix, float *dLdS, float *loss, int sms,
                      cudaStream_t s) {
    k_zero1<<<1, 1, 0, s>>>(loss);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || npix <= 0) return e;
    int64_t blocks = (npix + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    k_l1<<<(unsigned)blocks, 256, 0, s>>>(S, T, npix, (float)(1.0 / (double)npix), dLdS, loss);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sdgr
