// sdgr_internal.cuh -- device-side data layout and shared arithmetic of the
// B300 SAR Gaussian rasterizer.  Internal to libsdgr.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sdgr.h"

namespace sdgr {

constexpr int TILE = 16;         // tile edge (pixels); one CTA per tile
constexpr int TILE_PIX = TILE * TILE;
constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr int SORT_IPB = 2048;   // items per radix-sort block
constexpr int SORT_THREADS = 256;
constexpr int SCAN_IPB = 4096;   // items per scan block
constexpr int SCAN_THREADS = 256;

// Checked build (-DSDGR_CHECKED, libsdgr_checked.so): the stages that produce
// indices verify each one against its buffer; a bad index records
// SDGR_ERR_BOUNDS in the status word (the first error wins) and the access is
// skipped.  Nothing traps.  In the default build the checks compile away.
#ifdef SDGR_CHECKED
#define SDGR_IN_BOUNDS(st, cond) ::sdgr::check_bounds((st), (cond))
#else
#define SDGR_IN_BOUNDS(st, cond) true
#endif

// log2(e)
constexpr float LOG2E = 1.4426950408889634f;

// Per-view constants, written once per call by the plan upload.
struct alignas(16) ViewDev {
    float r[3][4];      // rows of R_r (float32): azimuth axis, elevation axis, line of sight
    double r2d[3];      // line-of-sight row in float64 (depth key)
    double cd[3];       // beam centre, float64
    float c[3];         // beam centre, float32
    float inv_dA;       // 1 / dA
    float inv_cy;       // 1 / (dR tan(theta)) : computation-plane cell height
    float inv_dR;       // 1 / dR
    float offx, offy;   // NA/2 - 1/2, NR/2 - 1/2
    int32_t NA, NR, tiles_x, tiles_y;
    int32_t scene, N;   // scene index and its Gaussian count
    int64_t g_off;      // first Gaussian of the scene in the parameter array
    int64_t vg_off;     // first (view, Gaussian) slot of this view
    int64_t pix_off;    // first pixel of this view in the image array
    int32_t tile_off;   // first tile of this view (per plane)
    int32_t sblk_off;   // first depth-sort block of this view
    int32_t sblk_n;     // depth-sort blocks of this view
    int32_t pad;
    float Ysh[16];      // real SH (degrees 1..3) of the direction toward the radar; 0 past the degree
};
static_assert(sizeof(ViewDev) == 256, "ViewDev layout");

struct alignas(16) SceneDev {
    int64_t g_off;      // first Gaussian
    int32_t N;          // Gaussian count
    int32_t vstart;     // first entry in the scene->view list
    int32_t vcount;     // views of this scene
    int32_t pad[3];
};
static_assert(sizeof(SceneDev) == 32, "SceneDev layout");

struct alignas(16) StatusDev {
    int32_t code;       // sdgr_status of the device side
    int32_t pad;
    int64_t required;   // instances the last bin/sort needed
    int64_t n_inst;     // instances emitted by the last bin/sort (if it fitted)
    int64_t pad2;
    unsigned long long pairs[2];  // sdgr_count_pairs: in-cutoff pairs per plane
};

// Work list of the raster kernels, rebuilt by every bin/sort: per plane the
// tiles with a non-empty instance list, view by view, and inside a view the
// longest lists first (longest-processing-time order by the bit length of
// the list size).  Per (plane, view, bucket) counters live in a separate
// array of 2 x V x 32 entries.
struct alignas(16) TileWorkDev {
    int32_t count[2];     // non-empty tiles per plane
    int32_t next[4];      // item counters of the persistent launches (K3, K4, K5, K6)
    int32_t pad[2];
};

// How a raster launch maps CTAs to tiles.  order == nullptr: CTA i takes tile
// i of the plane.  Otherwise CTAs take items of the plane's work list: one CTA
// per item (persistent_grid == 0) or persistent_grid CTAs that pull items
// from next[slot] until the list is exhausted.
struct TileSched {
    const int32_t *order;   // work list of this plane (tile indices, plane-local)
    TileWorkDev *work;
    int plane;              // 0 computation, 1 imaging
    int slot;               // item counter used by this launch
    int persistent_grid;    // > 0: persistent launch with this many CTAs
    int ntiles;             // tiles of the plane (bound of every work-list entry)
    int nb;                 // Gaussian records staged per batch (a supported size of the kernel)
};

// Staging batch sizes each raster kernel is built for (records per CTA
// batch): 0 intensity pass, 1 splat, 2 splat adjoint, 3 intensity adjoint.
// The first entry of each list is the kernel's default.
int stage_batch_options(int kernel, const int **sizes);

// One segment of a segmented radix sort: items [start, start + len), digits
// taken from (key - key_base); blk_start = first block of the segment.
#ifdef SDGR_CHECKED
__device__ __forceinline__ bool check_bounds(const StatusDev *st, bool ok) {
    if (!ok) atomicCAS(const_cast<int32_t *>(&st->code), (int32_t)SDGR_OK, (int32_t)SDGR_ERR_BOUNDS);
    return ok;
}
#endif

struct alignas(16) SegDev {
    uint32_t start, len, key_base, blk_start;
};

// Computation-plane record of one (view, Gaussian).  The conic is stored
// pre-scaled so that exp(-delta/2) = exp2(qa dx^2 + qb dx dy + qc dy^2):
// qa = -log2e/2 C00, qb = -log2e C01, qc = -log2e/2 C11.  ry is the
// half-height (pixels) of the K-ellipse's bounding box, with the same margin
// as the tile rectangles, so a kernel can skip rows the ellipse misses.
struct alignas(16) CompRec {
    float ux, uy, qa, qb;
    float qc, o, P, ry;
};

// Imaging-plane record: centre, pre-scaled conic, normaliser c_i, ry.
struct alignas(16) ImgRec {
    float ux, uy, qa, qb;
    float qc, cn, ry, pad1;
};

// Binning record of one (view, Gaussian) slot, written by preprocessing and
// read by the count gather and the instance emission in depth order (a
// random gather): one 32-byte sector per slot.  rc / ri: the tile
// rectangles (x0 | x1 << 16, y0 | y1 << 16) on the computation and imaging
// planes; mc / mi: for rectangles of at most 32 tiles, the tiles the
// K-ellipse reaches (bit i: the i-th tile of the rectangle, row by row);
// nc / ni: the slot's instance counts.
struct alignas(32) BinRec {
    uint2 rc, ri;
    uint32_t mc, mi, nc, ni;
};
static_assert(sizeof(BinRec) == 32, "BinRec layout");

// Half-height of the K-ellipse's bounding box for a 2D covariance whose yy
// entry is syy (same margin as the tile rectangles).
__device__ __forceinline__ float ellipse_ry(float syy, float K) { return K * sqrtf(syy) * 1.0001f + 1e-3f; }

// softplus(x) = log(1 + e^x) = -log(1 - sigmoid(x)): the optical depth of the
// Beer-Lambert opacity (alpha_mode 1).
__device__ __forceinline__ float softplus(float x) { return x > 0.f ? x + log1pf(expf(-x)) : log1pf(expf(x)); }

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// exp2 argument of the Gaussian weight at offset (dx, dy), with explicit
// round-to-nearest intrinsics.  Used by the pair-count diagnostic; the raster
// kernels evaluate the same quadratic in tile-local polynomial form.
__device__ __forceinline__ float gauss_q(float qa, float qb, float qc, float dx, float dy) {
    float t = __fmul_rn(qa, dx);
    t = __fmaf_rn(qb, dy, t);
    float u = __fmul_rn(qc, dy);
    u = __fmul_rn(u, dy);
    return __fmaf_rn(t, dx, u);
}

// Binary search: last index k in [0, n) with key(k) <= x (keys ascending,
// key(0) <= x).
template <typename F>
__device__ __forceinline__ int upper_index(int n, int64_t x, F key) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (key(mid) <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int view_of_vg(const ViewDev *views, int V, int64_t vg) {
    return upper_index(V, vg, [&](int k) { return views[k].vg_off; });
}

__device__ __forceinline__ int view_of_tile(const ViewDev *views, int V, int64_t tile) {
    return upper_index(V, tile, [&](int k) { return (int64_t)views[k].tile_off; });
}

__device__ __forceinline__ int view_of_sblk(const ViewDev *views, int V, int64_t b) {
    return upper_index(V, b, [&](int k) { return (int64_t)views[k].sblk_off; });
}

__device__ __forceinline__ uint32_t float_order_key(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// ---------------------------------------------------------------------------
// Launch wrappers (defined in the kernel translation units).
// ---------------------------------------------------------------------------
// Counts kernel launches (sdgr_launch_count); called after every launch.
void note_launch();

cudaError_t launch_upload(const void *host_src, size_t bytes, void *dev_dst, cudaStream_t s);

cudaError_t launch_preprocess(const float4 *params, const float4 *sh, int sh_count, const ViewDev *views, int V,
                              int64_t VG, float K, float eps, int norm_mode, int alpha_mode, CompRec *comp, ImgRec *img,
                              BinRec *bin, uint32_t *dkey, uint32_t *dval, int sms, cudaStream_t s);

// exclusive scans (scratch: see scan_scratch_elems)
size_t scan_scratch_elems(int64_t n);
cudaError_t launch_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *scratch, cudaStream_t s);
cudaError_t launch_scan_u64(const unsigned long long *in, unsigned long long *out, int64_t n,
                            unsigned long long *scratch, cudaStream_t s);

// radix sort passes
cudaError_t launch_depth_sort(const ViewDev *views, int V, int nblocks, SegDev *segs, uint32_t *k0, uint32_t *v0,
                              uint32_t *k1, uint32_t *v1, uint32_t *hist, uint32_t *scan_scratch, cudaStream_t s);
cudaError_t launch_inst_sort(const StatusDev *st, const unsigned long long *soff, const unsigned long long *scnt,
                             int64_t VG, const ViewDev *views, int V, int tiles, int64_t cap, int key_bits,
                             SegDev *segs, uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, uint32_t *hist,
                             uint32_t *scan_scratch, int *final_in_1, cudaStream_t s);
cudaError_t launch_gather_counts(const uint32_t *sorted_vg, const BinRec *bin, int64_t VG, unsigned long long *scnt,
                                 int sms, cudaStream_t s);
cudaError_t launch_check_capacity(const unsigned long long *scnt, const unsigned long long *soff, int64_t VG,
                                  int64_t cap, StatusDev *st, cudaStream_t s);
cudaError_t launch_emit(const uint32_t *sorted_vg, const unsigned long long *soff, const unsigned long long *scnt,
                        const BinRec *bin, const ViewDev *views, int V, int64_t VG,
                        int total_tiles, const StatusDev *st, int64_t cap, uint32_t *keys, uint32_t *vals, int sms,
                        cudaStream_t s);
// vhist, voff: 2 * V * 32 entries; vt, vbase: 2 * V; scratch:
// scan_scratch_elems(2 * V) entries.
cudaError_t launch_tile_order(const uint2 *ranges, int tiles, const ViewDev *views, int V, TileWorkDev *work,
                              int32_t *order, uint32_t *vhist, uint32_t *voff, uint32_t *vt, uint32_t *vbase,
                              uint32_t *scratch, int sms, cudaStream_t s);
cudaError_t launch_ranges(const uint32_t *keys, StatusDev *st, int64_t cap, int64_t nranges, uint2 *ranges, int sms,
                          cudaStream_t s);

// raster passes
cudaError_t launch_intensity_fwd(const uint2 *ranges, const uint32_t *vals, const CompRec *comp, const ViewDev *views,
                                 int V, int tiles, float cut, float Tfloor, int alpha_mode, const StatusDev *st, float *A,
                                 float *Tend, int32_t *last, const TileSched &sched, cudaStream_t s);
cudaError_t launch_splat_fwd(const uint2 *rangesI, const uint32_t *vals, const ImgRec *img, const CompRec *comp,
                             const float *A, const ViewDev *views, int V, int tiles, float cut, const StatusDev *st,
                             float *images, const TileSched &sched, cudaStream_t s);
cudaError_t launch_splat_bwd(const uint2 *rangesI, const uint32_t *vals, const ImgRec *img, const float *dLdS,
                             const ViewDev *views, int V, int tiles, float cut, const StatusDev *st, float4 *accI,
                             const TileSched &sched, cudaStream_t s);
cudaError_t launch_intensity_bwd(const uint2 *ranges, const uint32_t *vals, const CompRec *comp, const ImgRec *img,
                                 const float4 *accI, const float *Tend, const int32_t *last, const ViewDev *views,
                                 int V, int tiles, float cut, int alpha_mode, const StatusDev *st, float4 *accC,
                                 const TileSched &sched, cudaStream_t s);
// CTAs per SM of a raster kernel at 256 threads (occupancy query, cached).
int raster_blocks_per_sm(int kernel, int nb);
cudaError_t launch_count_pairs(const uint2 *ranges, const uint32_t *vals, const CompRec *comp, const ImgRec *img,
                               const ViewDev *views, int V, int tiles, float cut, StatusDev *st, cudaStream_t s);
cudaError_t launch_intensity_out(const CompRec *comp, const float *A, int64_t VG, float *I, int sms, cudaStream_t s);
cudaError_t launch_selfcheck(uint32_t *flags, cudaStream_t s);
// sink: 1024 floats; cycles: one counter, zeroed by the caller.
cudaError_t launch_pipe_rate(int op, int iters, float *sink, unsigned long long *cycles, int *blocks_per_sm,
                             int sms, cudaStream_t s);

// parameter adjoint, optimiser, loss
cudaError_t launch_param_bwd(const float4 *params, const ViewDev *views, const SceneDev *scenes,
                             const int32_t *scene_views, int n_scenes, int64_t n_gauss, float eps, int norm_mode,
                             int alpha_mode,
                             const float *A, const CompRec *comp, const float4 *accI, const float4 *accC,
                             const StatusDev *st, float4 *grads, float4 *dsh, float *dens_accum,
                             float *dens_count, int sms, cudaStream_t s);
cudaError_t launch_adam(float4 *p, const float4 *g, float4 *m, float4 *v, int64_t n4, const float *lr, float b1,
                        float b2, float eps, int step, int sms, cudaStream_t s);
cudaError_t launch_adam_dev(float4 *p, const float4 *g, float4 *m, float4 *v, int64_t n4, const float *lr, float b1,
                            float b2, float eps, int32_t *step, int sms, cudaStream_t s);
cudaError_t launch_l1(const float *S, const float *T, int64_t npix, float *dLdS, float *loss, int sms,
                      cudaStream_t s);

}  // namespace sdgr
