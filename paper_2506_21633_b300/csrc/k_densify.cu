// k_densify.cu -- densification and pruning of the Gaussian set (Section
// II-B "Densification and Pruning Operation", thresholds of Section III-D):
// a classification pass (keep / clone / split / prune, one count per
// Gaussian), an exclusive scan of the counts, and an emission pass that
// writes the survivors in order with their parameters, optimiser moments and
// SH coefficients.  All decisions are float32 comparisons against
// thresholds that the host converts once (log / logit in float64, then
// rounded).
#include "sdgr_internal.cuh"

namespace sdgr {

enum : uint32_t { ACT_PRUNE = 0, ACT_KEEP = 1, ACT_CLONE = 2, ACT_SPLIT = 3 };

struct DensifyThresholds {
    float grad;          // mean |dL/du_I| threshold
    float log_dense;     // ln(dense_scale)
    float log_max;       // ln(max_scale)
    float logit_min_o;   // logit(min_opacity)
    float min_P;
    float log_split;     // ln(split_factor)
};

__global__ void __launch_bounds__(256)
k_densify_classify(const float4 *__restrict__ params, const float *__restrict__ accum, const float *__restrict__ count,
                   int64_t N, DensifyThresholds th, uint32_t *__restrict__ act, uint32_t *__restrict__ cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const float4 p0 = params[3 * i], p1 = params[3 * i + 1];
        const float lsmax = fmaxf(p1.x, fmaxf(p1.y, p1.z));
        uint32_t a = ACT_KEEP;
        if (p0.w < th.logit_min_o || p1.w < th.min_P || lsmax > th.log_max) {
            a = ACT_PRUNE;
        } else {
            const float c = count[i];
            if (c > 0.f && __fdiv_rn(accum[i], c) > th.grad) a = lsmax <= th.log_dense ? ACT_CLONE : ACT_SPLIT;
        }
        act[i] = a;
        cnt[i] = a == ACT_PRUNE ? 0u : (a == ACT_KEEP ? 1u : 2u);
    }
}

__device__ __forceinline__ void write_row(float *dst, int64_t k, int w, const float *src) {
    for (int j = 0; j < w; ++j) dst[k * w + j] = src[j];
}

__global__ void __launch_bounds__(256)
k_densify_emit(const float *__restrict__ params, const float *__restrict__ grads, const float *__restrict__ m,
               const float *__restrict__ v, const float *__restrict__ sh, int64_t N, DensifyThresholds th,
               const uint32_t *__restrict__ act, const uint32_t *__restrict__ off, float *__restrict__ op,
               float *__restrict__ om, float *__restrict__ ov, float *__restrict__ osh) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float zero[12] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const uint32_t a = act[i];
        if (a == ACT_PRUNE) continue;
        const int64_t k = off[i];
        const float *pi = params + 12 * i;
        if (a == ACT_KEEP || a == ACT_CLONE) {
            write_row(op, k, 12, pi);
            write_row(om, k, 12, m + 12 * i);
            write_row(ov, k, 12, v + 12 * i);
            if (sh) write_row(osh, k, 16, sh + 16 * i);
        }
        // direction -dL/dmu (zero if the gradient vanishes)
        const float gx = grads[12 * i], gy = grads[12 * i + 1], gz = grads[12 * i + 2];
        const float gn = sqrtf(gx * gx + gy * gy + gz * gz);
        const float ux = gn > 0.f ? -gx / gn : 0.f, uy = gn > 0.f ? -gy / gn : 0.f, uz = gn > 0.f ? -gz / gn : 0.f;
        // largest scale and its axis (a column of R(q))
        int ax = 0;
        if (pi[5] > pi[4 + ax]) ax = 1;
        if (pi[6] > pi[4 + ax]) ax = 2;
        const float smax = expf(pi[4 + ax]);
        if (a == ACT_CLONE) {
            float row[12];
            for (int j = 0; j < 12; ++j) row[j] = pi[j];
            row[0] += smax * ux;
            row[1] += smax * uy;
            row[2] += smax * uz;
            write_row(op, k + 1, 12, row);
            write_row(om, k + 1, 12, zero);
            write_row(ov, k + 1, 12, zero);
            if (sh) write_row(osh, k + 1, 16, sh + 16 * i);
        } else if (a == ACT_SPLIT) {
            const float qn = 1.0f / sqrtf(pi[8] * pi[8] + pi[9] * pi[9] + pi[10] * pi[10] + pi[11] * pi[11]);
            const float w = pi[8] * qn, x = pi[9] * qn, y = pi[10] * qn, z = pi[11] * qn;
            float e[3];
            if (ax == 0) { e[0] = 1.f - 2.f * (y * y + z * z); e[1] = 2.f * (x * y + w * z); e[2] = 2.f * (x * z - w * y); }
            else if (ax == 1) { e[0] = 2.f * (x * y - w * z); e[1] = 1.f - 2.f * (x * x + z * z); e[2] = 2.f * (y * z + w * x); }
            else { e[0] = 2.f * (x * z + w * y); e[1] = 2.f * (y * z - w * x); e[2] = 1.f - 2.f * (x * x + y * y); }
            const float sgn = (e[0] * ux + e[1] * uy + e[2] * uz) < 0.f ? -1.f : 1.f;  // child 0 toward -dL/dmu
            for (int c = 0; c < 2; ++c) {
                float row[12];
                for (int j = 0; j < 12; ++j) row[j] = pi[j];
                const float d = (c == 0 ? 0.5f : -0.5f) * sgn * smax;
                row[0] += d * e[0];
                row[1] += d * e[1];
                row[2] += d * e[2];
                row[4] -= th.log_split;
                row[5] -= th.log_split;
                row[6] -= th.log_split;
                write_row(op, k + c, 12, row);
                write_row(om, k + c, 12, zero);
                write_row(ov, k + c, 12, zero);
                if (sh) write_row(osh, k + c, 16, sh + 16 * i);
            }
        }
    }
}

cudaError_t launch_densify_classify(const float4 *params, const float *accum, const float *count, int64_t N,
                                    const DensifyThresholds &th, uint32_t *act, uint32_t *cnt, int sms,
                                    cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    int64_t blocks = (N + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    k_densify_classify<<<(unsigned)blocks, 256, 0, s>>>(params, accum, count, N, th, act, cnt);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_densify_emit(const float *params, const float *grads, const float *m, const float *v,
                                const float *sh, int64_t N, const DensifyThresholds &th, const uint32_t *act,
                                const uint32_t *off, float *op, float *om, float *ov, float *osh, int sms,
                                cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    int64_t blocks = (N + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    k_densify_emit<<<(unsigned)blocks, 256, 0, s>>>(params, grads, m, v, sh, N, th, act, off, op, om, ov, osh);
    note_launch();
    return cudaGetLastError();
}

}  // namespace sdgr

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
using namespace sdgr;

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

extern "C" size_t sdgr_densify_scratch_bytes(int64_t N) {
    if (N < 0) return 0;
    return 2 * align256((size_t)N * 4 + 16) + align256(scan_scratch_elems(N) * 4 + 16);
}

extern "C" sdgr_status sdgr_densify(const float *params, const float *grads, const float *accum, const float *count,
                                    const float *m, const float *v, const float *sh, int64_t N,
                                    const sdgr_densify_cfg *cfg, float *out_params, float *out_m, float *out_v,
                                    float *out_sh, int64_t out_capacity, void *scratch, int64_t *new_N,
                                    void *stream) {
    if (!cfg || !new_N || N < 0 || out_capacity < 0 || (N > 0 && (!params || !grads || !accum || !count || !m ||
                                                                    !v || !scratch)))
        return SDGR_ERR_INVALID;
    if ((sh != nullptr) != (out_sh != nullptr)) return SDGR_ERR_INVALID;
    if (!(cfg->split_factor > 1.f) || !(cfg->dense_scale > 0.f) || !(cfg->max_scale > 0.f) ||
        !(cfg->min_opacity > 0.f && cfg->min_opacity < 1.f))
        return SDGR_ERR_INVALID;
    if (((uintptr_t)params | (uintptr_t)scratch) % 16 != 0) return SDGR_ERR_INVALID;
    *new_N = 0;
    if (N == 0) return SDGR_OK;
    DensifyThresholds th;
    th.grad = cfg->grad_threshold;
    th.log_dense = (float)log((double)cfg->dense_scale);
    th.log_max = (float)log((double)cfg->max_scale);
    th.logit_min_o = (float)(log((double)cfg->min_opacity) - log1p(-(double)cfg->min_opacity));
    th.min_P = cfg->min_P;
    th.log_split = (float)log((double)cfg->split_factor);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(scratch);
    uint32_t *act = reinterpret_cast<uint32_t *>(base);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(base + align256((size_t)N * 4 + 16));
    uint32_t *scr = reinterpret_cast<uint32_t *>(base + 2 * align256((size_t)N * 4 + 16));
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SDGR_ERR_CUDA;
    if (launch_densify_classify(reinterpret_cast<const float4 *>(params), accum, count, N, th, act, cnt, sms, s) !=
        cudaSuccess)
        return SDGR_ERR_CUDA;
    uint32_t last_cnt = 0, last_off = 0;
    // offsets in place of the counts' copy: scan cnt -> act2 is not needed; keep counts for the total
    if (cudaMemcpyAsync(&last_cnt, cnt + (N - 1), 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return SDGR_ERR_CUDA;
    if (launch_scan_u32(cnt, cnt, N, scr, s) != cudaSuccess) return SDGR_ERR_CUDA;
    if (cudaMemcpyAsync(&last_off, cnt + (N - 1), 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return SDGR_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SDGR_ERR_CUDA;
    const int64_t total = (int64_t)last_off + last_cnt;
    *new_N = total;
    if (total > out_capacity) return SDGR_ERR_CAPACITY;
    if (!out_params || !out_m || !out_v) return SDGR_ERR_INVALID;
    if (launch_densify_emit(params, grads, m, v, sh, N, th, act, cnt, out_params, out_m, out_v, out_sh, sms, s) !=
        cudaSuccess)
        return SDGR_ERR_CUDA;
    return SDGR_OK;
}
