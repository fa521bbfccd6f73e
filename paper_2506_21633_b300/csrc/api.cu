// api.cu -- host side of the C ABI declared in include/sdgr.h: argument
// validation, the per-call plan (view / scene tables), the workspace layout
// inside the caller's device buffer, and the launch sequence of each step.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <vector>

#include "sdgr_internal.cuh"

using namespace sdgr;

static std::atomic<long long> g_launches{0};

void sdgr::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {

constexpr size_t ALIGN = 256;
constexpr int64_t MAX_INSTANCES = (int64_t)0x7fffffff;  // instance indices are 32-bit

struct Layout {
    size_t views, scenes, scene_views, status;
    size_t comp, img, bin;
    size_t dk0, dv0, dk1, dv1;
    size_t scnt, soff, scan64;
    size_t ik0, iv0, ik1, iv1;
    size_t hist, scan32, ranges, segs, order, work, vhist, voff, vt, vbase, vscan;
    size_t A, Tend, last, accI, accC;
    size_t total;
};

size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

bool caps_ok(const sdgr_caps *c) {
    return c && c->max_views >= 0 && c->max_scenes >= 0 && c->max_gaussians >= 0 && c->max_view_gauss >= 0 &&
           c->max_pixels >= 0 && c->max_tiles >= 0 && c->max_instances >= 0 && c->max_instances <= MAX_INSTANCES &&
           c->max_view_gauss < ((int64_t)1 << 32) && c->max_tiles < ((int64_t)1 << 30) &&
           c->max_views < (1 << 24) && c->max_pixels < ((int64_t)1 << 40) && c->max_gaussians < ((int64_t)1 << 34);
}

int64_t depth_sort_blocks_cap(const sdgr_caps *c) { return c->max_view_gauss / SORT_IPB + c->max_views + 1; }

Layout make_layout(const sdgr_caps *c) {
    Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align_up(bytes > 0 ? bytes : 1);
        return o;
    };
    const size_t VG = (size_t)c->max_view_gauss, V = (size_t)c->max_views, S = (size_t)c->max_scenes;
    const size_t NI = (size_t)c->max_instances, NP = (size_t)c->max_pixels, NT = (size_t)c->max_tiles;
    L.views = take(V * sizeof(ViewDev));
    L.scenes = take(S * sizeof(SceneDev));
    L.scene_views = take(V * sizeof(int32_t));
    L.status = take(sizeof(StatusDev));
    L.comp = take(VG * sizeof(CompRec));
    L.img = take(VG * sizeof(ImgRec));
    L.bin = take(VG * sizeof(BinRec));
    L.dk0 = take(VG * 4);
    L.dv0 = take(VG * 4);
    L.dk1 = take(VG * 4);
    L.dv1 = take(VG * 4);
    L.scnt = take(2 * VG * 8);
    L.soff = take(2 * VG * 8);
    L.scan64 = take(scan_scratch_elems((int64_t)(2 * VG)) * 8);
    L.ik0 = take(NI * 4);
    L.iv0 = take(NI * 4);
    L.ik1 = take(NI * 4);
    L.iv1 = take(NI * 4);
    int64_t hb = depth_sort_blocks_cap(c);
    int64_t ib = (c->max_instances + SORT_IPB - 1) / SORT_IPB + 2 * (int64_t)c->max_views;
    int64_t hn = (hb > ib ? hb : ib) * RADIX;
    L.hist = take((size_t)hn * 4);
    L.scan32 = take(scan_scratch_elems(hn) * 4);
    L.ranges = take(2 * NT * sizeof(uint2));
    L.segs = take((2 * V + 2) * sizeof(SegDev));
    L.order = take(2 * NT * 4);
    L.work = take(sizeof(TileWorkDev));
    L.vhist = take(2 * V * 32 * 4);
    L.voff = take(2 * V * 32 * 4);
    L.vt = take(2 * V * 4);
    L.vbase = take(2 * V * 4);
    L.vscan = take(scan_scratch_elems((int64_t)(2 * V)) * 4);
    L.A = take(VG * 4);
    L.Tend = take(NP * 4);
    L.last = take(NP * 4);
    L.accI = take(VG * 2 * sizeof(float4));
    L.accC = take(VG * 2 * sizeof(float4));
    L.total = off;
    return L;
}

bool cfg_ok(const sdgr_cfg *cfg) {
    return cfg && cfg->cutoff_K > 0.f && isfinite(cfg->cutoff_K) && cfg->dilation_eps >= 0.f &&
           isfinite(cfg->dilation_eps) && cfg->T_min >= 0.f && cfg->T_min < 1.f &&
           (cfg->norm_mode == 0 || cfg->norm_mode == 1) && (cfg->alpha_mode == 0 || cfg->alpha_mode == 1);
}

bool view_ok(const sdgr_view &v) {
    const double half_pi = 1.5707963267948966;
    return v.theta > 0.0 && v.theta < half_pi && v.dA > 0.0 && v.dR > 0.0 && isfinite(v.phi) && isfinite(v.dA) &&
           isfinite(v.dR) && v.NA > 0 && v.NR > 0 && v.NA <= (1 << 20) && v.NR <= (1 << 20) &&
           isfinite(v.center[0]) && isfinite(v.center[1]) && isfinite(v.center[2]);
}

int tiles_of(int n) { return (n + TILE - 1) / TILE; }

}  // namespace

struct sdgr_ws {
    char *base = nullptr;
    size_t bytes = 0;
    sdgr_cfg cfg;
    sdgr_caps caps;
    Layout L;
    int sms = 148;
    // plan of the last sdgr_preprocess()
    int V = 0, n_scenes = 0;
    int64_t VG = 0, npix = 0, n_gauss = 0;
    int tiles = 0, sort_blocks = 0, key_bits = 0;
    const float *params = nullptr;
    int stage = 0;  // 1 preprocessed, 2 sorted, 3 forward done
    uint32_t *inst_keys = nullptr, *inst_vals = nullptr;
    // stage timing (sdgr_profile_enable / sdgr_profile_read)
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;      // pool, two per recorded launch
    std::vector<int> prof_stage;           // stage of each recorded pair
    int prof_used = 0;
    double prof_ms[SDGR_NUM_STAGES] = {0};
    int64_t prof_n[SDGR_NUM_STAGES] = {0};
    const float *sh = nullptr;  // sdgr_set_sh
    float *dsh = nullptr;
    int sh_degree = 0;
    float *dens_accum = nullptr, *dens_count = nullptr;  // sdgr_set_densify_stats
    int sched = SDGR_SCHED_ORDERED | SDGR_SCHED_PERSISTENT;  // sdgr_set_schedule
    int stage_batch[4] = {0, 0, 0, 0};  // sdgr_set_stage_batch (0: the kernel's default)
    std::vector<ViewDev> hviews;
    std::vector<SceneDev> hscenes;
    std::vector<int32_t> hscene_views;

    template <typename T>
    T *at(size_t off) const {
        return reinterpret_cast<T *>(base + off);
    }
};

namespace {

constexpr int PROF_PAIRS = 2048;

cudaError_t prof_harvest(sdgr_ws *ws) {
    if (ws->prof_used == 0) return cudaSuccess;
    cudaError_t e = cudaEventSynchronize(ws->prof_ev[2 * (ws->prof_used - 1) + 1]);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < ws->prof_used; ++k) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, ws->prof_ev[2 * k], ws->prof_ev[2 * k + 1]);
        if (e != cudaSuccess) return e;
        ws->prof_ms[ws->prof_stage[k]] += ms;
        ws->prof_n[ws->prof_stage[k]] += 1;
    }
    ws->prof_used = 0;
    return cudaSuccess;
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

// Stage events.  On a stream that is being captured into a CUDA graph they
// become event-record nodes of the graph (recorded again by every replay),
// so the stage times of a replay are read after it has run.
void prof_record(cudaEvent_t e, cudaStream_t s) {
    if (capturing(s))
        cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
        cudaEventRecord(e, s);
}

// Records the start event of a stage; returns the pair index or -1.
int prof_begin(sdgr_ws *ws, int stage, cudaStream_t s) {
    if (!ws->prof_on) return -1;
    if (ws->prof_used == PROF_PAIRS && (capturing(s) || prof_harvest(ws) != cudaSuccess)) return -1;
    const int k = ws->prof_used++;
    ws->prof_stage[k] = stage;
    prof_record(ws->prof_ev[2 * k], s);
    return k;
}

void prof_end(sdgr_ws *ws, int k, cudaStream_t s) {
    if (k >= 0) prof_record(ws->prof_ev[2 * k + 1], s);
}

}  // namespace

#define CK(call)                                      \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return SDGR_ERR_CUDA;  \
    } while (0)

extern "C" {

const char *sdgr_status_string(sdgr_status s) {
    switch (s) {
        case SDGR_OK: return "ok";
        case SDGR_ERR_INVALID: return "invalid argument";
        case SDGR_ERR_CUDA: return "CUDA runtime error";
        case SDGR_ERR_CAPACITY: return "instance capacity exceeded";
        case SDGR_ERR_TIMEOUT: return "bounded device wait timed out";
        case SDGR_ERR_STATE: return "calls out of order on this workspace";
        case SDGR_ERR_BOUNDS: return "checked build: an index left its buffer";
    }
    return "unknown status";
}

sdgr_status sdgr_caps_for(const sdgr_view *views, int32_t V, const int64_t *scene_offsets, int32_t n_scenes,
                          int64_t instances, sdgr_caps *out) {
    if (!out || V < 0 || n_scenes < 0 || (V > 0 && !views) || !scene_offsets || instances < 0 ||
        instances > MAX_INSTANCES)
        return SDGR_ERR_INVALID;
    if (scene_offsets[0] != 0) return SDGR_ERR_INVALID;
    for (int s = 0; s < n_scenes; ++s)
        if (scene_offsets[s + 1] < scene_offsets[s]) return SDGR_ERR_INVALID;
    int64_t vg = 0, pix = 0, tiles = 0;
    for (int v = 0; v < V; ++v) {
        if (!view_ok(views[v]) || views[v].scene < 0 || views[v].scene >= n_scenes) return SDGR_ERR_INVALID;
        vg += scene_offsets[views[v].scene + 1] - scene_offsets[views[v].scene];
        pix += (int64_t)views[v].NA * views[v].NR;
        tiles += (int64_t)tiles_of(views[v].NA) * tiles_of(views[v].NR);
    }
    out->max_views = V;
    out->max_scenes = n_scenes;
    out->max_gaussians = scene_offsets[n_scenes];
    out->max_view_gauss = vg;
    out->max_pixels = pix;
    out->max_tiles = tiles;
    out->max_instances = instances;
    return caps_ok(out) ? SDGR_OK : SDGR_ERR_INVALID;
}

sdgr_status sdgr_workspace_size(const sdgr_cfg *cfg, const sdgr_caps *caps, size_t *bytes) {
    if (!bytes || !cfg_ok(cfg) || !caps_ok(caps)) return SDGR_ERR_INVALID;
    *bytes = make_layout(caps).total;
    return SDGR_OK;
}

sdgr_status sdgr_ws_create(sdgr_ws **out, void *device_buffer, size_t bytes, const sdgr_cfg *cfg,
                           const sdgr_caps *caps) {
    if (!out || !device_buffer || !cfg_ok(cfg) || !caps_ok(caps)) return SDGR_ERR_INVALID;
    if (((uintptr_t)device_buffer) % ALIGN != 0) return SDGR_ERR_INVALID;
    Layout L = make_layout(caps);
    if (bytes < L.total) return SDGR_ERR_INVALID;
    sdgr_ws *ws = new (std::nothrow) sdgr_ws();
    if (!ws) return SDGR_ERR_INVALID;
    ws->base = static_cast<char *>(device_buffer);
    ws->bytes = bytes;
    ws->cfg = *cfg;
    ws->caps = *caps;
    ws->L = L;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&ws->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete ws;
        return SDGR_ERR_CUDA;
    }
    *out = ws;
    return SDGR_OK;
}

sdgr_status sdgr_ws_destroy(sdgr_ws *ws) {
    if (!ws) return SDGR_ERR_INVALID;
    for (cudaEvent_t e : ws->prof_ev) cudaEventDestroy(e);
    delete ws;
    return SDGR_OK;
}

sdgr_status sdgr_preprocess(sdgr_ws *ws, const float *params, const int64_t *scene_offsets, int32_t n_scenes,
                            const sdgr_view *views, int32_t V, void *stream) {
    if (!ws || !scene_offsets || n_scenes < 0 || V < 0 || (V > 0 && !views)) return SDGR_ERR_INVALID;
    if (n_scenes > ws->caps.max_scenes || V > ws->caps.max_views) return SDGR_ERR_INVALID;
    if (scene_offsets[0] != 0) return SDGR_ERR_INVALID;
    for (int s = 0; s < n_scenes; ++s)
        if (scene_offsets[s + 1] < scene_offsets[s]) return SDGR_ERR_INVALID;
    const int64_t n_gauss = scene_offsets[n_scenes];
    if (n_gauss > ws->caps.max_gaussians) return SDGR_ERR_INVALID;
    if (n_gauss > 0 && (!params || ((uintptr_t)params) % 16 != 0)) return SDGR_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // plan: per-view offsets and constants
    ws->hviews.assign((size_t)V, ViewDev());
    int64_t vg = 0, pix = 0;
    int64_t tiles = 0, sblk = 0;
    for (int v = 0; v < V; ++v) {
        const sdgr_view &in = views[v];
        if (!view_ok(in) || in.scene < 0 || in.scene >= n_scenes) return SDGR_ERR_INVALID;
        ViewDev &d = ws->hviews[v];
        memset(&d, 0, sizeof(d));
        const double sp = sin(in.phi), cp = cos(in.phi), st = sin(in.theta), ct = cos(in.theta);
        // R_r of eq. R_r: azimuth axis, elevation axis, line of sight
        const double Rr[3][3] = {{-sp, -cp, 0.0}, {-st * cp, st * sp, ct}, {-ct * cp, ct * sp, -st}};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) d.r[a][b] = (float)Rr[a][b];
        for (int b = 0; b < 3; ++b) {
            d.r2d[b] = Rr[2][b];
            d.cd[b] = in.center[b];
            d.c[b] = (float)in.center[b];
        }
        // real SH of degrees 1..3 at the direction toward the radar (float64, rounded)
        {
            const double x = ct * cp, y = -ct * sp, z = st, pi = 3.14159265358979323846;
            const double c1 = sqrt(3.0 / (4.0 * pi)), c2 = sqrt(15.0 / pi) / 2.0, c20 = sqrt(5.0 / pi) / 4.0;
            const double c22 = sqrt(15.0 / pi) / 4.0, c33 = sqrt(35.0 / (2.0 * pi)) / 4.0;
            const double c32 = sqrt(105.0 / pi) / 2.0, c31 = sqrt(21.0 / (2.0 * pi)) / 4.0, c30 = sqrt(7.0 / pi) / 4.0;
            const double Y[15] = {c1 * y, c1 * z, c1 * x,
                                  c2 * x * y, c2 * y * z, c20 * (3 * z * z - 1), c2 * x * z, c22 * (x * x - y * y),
                                  c33 * y * (3 * x * x - y * y), c32 * x * y * z, c31 * y * (5 * z * z - 1),
                                  c30 * z * (5 * z * z - 3), c31 * x * (5 * z * z - 1), 0.5 * c32 * z * (x * x - y * y),
                                  c33 * x * (x * x - 3 * y * y)};
            const int nk = ws->sh_degree <= 0 ? 0 : (ws->sh_degree == 1 ? 3 : (ws->sh_degree == 2 ? 8 : 15));
            for (int k = 0; k < 16; ++k) d.Ysh[k] = k < nk ? (float)Y[k] : 0.f;
        }
        d.inv_dA = (float)(1.0 / in.dA);
        d.inv_cy = (float)(1.0 / (in.dR * tan(in.theta)));
        d.inv_dR = (float)(1.0 / in.dR);
        d.offx = (float)(in.NA * 0.5 - 0.5);
        d.offy = (float)(in.NR * 0.5 - 0.5);
        d.NA = in.NA;
        d.NR = in.NR;
        d.tiles_x = tiles_of(in.NA);
        d.tiles_y = tiles_of(in.NR);
        d.scene = in.scene;
        const int64_t N = scene_offsets[in.scene + 1] - scene_offsets[in.scene];
        d.N = (int32_t)N;
        d.g_off = scene_offsets[in.scene];
        d.vg_off = vg;
        d.pix_off = pix;
        d.tile_off = (int32_t)tiles;
        d.sblk_off = (int32_t)sblk;
        d.sblk_n = (int32_t)((N + SORT_IPB - 1) / SORT_IPB);
        vg += N;
        pix += (int64_t)in.NA * in.NR;
        tiles += (int64_t)d.tiles_x * d.tiles_y;
        sblk += d.sblk_n;
        if (N >= ((int64_t)1 << 31)) return SDGR_ERR_INVALID;
    }
    if (vg > ws->caps.max_view_gauss || pix > ws->caps.max_pixels || tiles > ws->caps.max_tiles ||
        sblk > depth_sort_blocks_cap(&ws->caps))
        return SDGR_ERR_INVALID;
    // scenes and their view lists
    ws->hscenes.assign((size_t)n_scenes, SceneDev());
    ws->hscene_views.clear();
    for (int sc = 0; sc < n_scenes; ++sc) {
        SceneDev &d = ws->hscenes[sc];
        memset(&d, 0, sizeof(d));
        d.g_off = scene_offsets[sc];
        d.N = (int32_t)(scene_offsets[sc + 1] - scene_offsets[sc]);
        d.vstart = (int32_t)ws->hscene_views.size();
        for (int v = 0; v < V; ++v)
            if (views[v].scene == sc) ws->hscene_views.push_back(v);
        d.vcount = (int32_t)ws->hscene_views.size() - d.vstart;
    }
    while (ws->hscene_views.size() % 4) ws->hscene_views.push_back(0);

    ws->V = V;
    ws->n_scenes = n_scenes;
    ws->VG = vg;
    ws->npix = pix;
    ws->n_gauss = n_gauss;
    ws->tiles = (int)tiles;
    ws->sort_blocks = (int)sblk;
    int64_t max_view_tiles = 1;
    for (int v = 0; v < V; ++v)
        max_view_tiles = std::max<int64_t>(max_view_tiles, (int64_t)ws->hviews[v].tiles_x * ws->hviews[v].tiles_y);
    int bits = 1;
    while (((int64_t)1 << bits) < max_view_tiles) ++bits;
    ws->key_bits = bits;  // tile bits within one view: the instance sort is segmented per (plane, view)
    ws->params = params;
    ws->stage = 0;

    const Layout &L = ws->L;
    if (V > 0) CK(launch_upload(ws->hviews.data(), (size_t)V * sizeof(ViewDev), ws->base + L.views, s));
    if (n_scenes > 0) CK(launch_upload(ws->hscenes.data(), (size_t)n_scenes * sizeof(SceneDev), ws->base + L.scenes, s));
    if (!ws->hscene_views.empty())
        CK(launch_upload(ws->hscene_views.data(), ws->hscene_views.size() * 4, ws->base + L.scene_views, s));
    CK(cudaMemsetAsync(ws->base + L.status, 0, sizeof(StatusDev), s));
    const sdgr_cfg &c = ws->cfg;
    const int pk = prof_begin(ws, SDGR_STAGE_PREPROCESS, s);
    const int sh_count = ws->sh ? (ws->sh_degree <= 0 ? 0 : (ws->sh_degree == 1 ? 3 : (ws->sh_degree == 2 ? 8 : 15))) : 0;
    CK(launch_preprocess(reinterpret_cast<const float4 *>(params),
                         sh_count > 0 ? reinterpret_cast<const float4 *>(ws->sh) : nullptr, sh_count,
                         ws->at<ViewDev>(L.views), V, vg, c.cutoff_K,
                         c.dilation_eps, c.norm_mode, c.alpha_mode, ws->at<CompRec>(L.comp), ws->at<ImgRec>(L.img),
                         ws->at<BinRec>(L.bin), ws->at<uint32_t>(L.dk0), ws->at<uint32_t>(L.dv0), ws->sms, s));
    prof_end(ws, pk, s);
    ws->stage = 1;
    return SDGR_OK;
}

sdgr_status sdgr_bin_sort(sdgr_ws *ws, void *stream) {
    if (!ws) return SDGR_ERR_INVALID;
    if (ws->stage < 1) return SDGR_ERR_STATE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Layout &L = ws->L;
    StatusDev *st = ws->at<StatusDev>(L.status);
    const ViewDev *views = ws->at<ViewDev>(L.views);
    // depth order per view: stable radix sort of the keys, values = slot index
    const int pk0 = prof_begin(ws, SDGR_STAGE_DEPTH_SORT, s);
    CK(launch_depth_sort(views, ws->V, ws->sort_blocks, ws->at<SegDev>(L.segs), ws->at<uint32_t>(L.dk0),
                         ws->at<uint32_t>(L.dv0),
                         ws->at<uint32_t>(L.dk1), ws->at<uint32_t>(L.dv1), ws->at<uint32_t>(L.hist),
                         ws->at<uint32_t>(L.scan32), s));
    prof_end(ws, pk0, s);
    const int pk1 = prof_begin(ws, SDGR_STAGE_BIN, s);
    const uint32_t *sorted_vg = ws->at<uint32_t>(L.dv0);
    unsigned long long *scnt = ws->at<unsigned long long>(L.scnt);
    unsigned long long *soff = ws->at<unsigned long long>(L.soff);
    CK(launch_gather_counts(sorted_vg, ws->at<BinRec>(L.bin), ws->VG, scnt, ws->sms, s));
    CK(launch_scan_u64(scnt, soff, 2 * ws->VG, ws->at<unsigned long long>(L.scan64), s));
    CK(launch_check_capacity(scnt, soff, ws->VG, ws->caps.max_instances, st, s));
    CK(launch_emit(sorted_vg, soff, scnt, ws->at<BinRec>(L.bin), views, ws->V, ws->VG, ws->tiles,
                   st, ws->caps.max_instances, ws->at<uint32_t>(L.ik0), ws->at<uint32_t>(L.iv0), ws->sms, s));
    int final1 = 0;
    CK(launch_inst_sort(st, soff, scnt, ws->VG, views, ws->V, ws->tiles, ws->caps.max_instances, ws->key_bits,
                        ws->at<SegDev>(L.segs), ws->at<uint32_t>(L.ik0), ws->at<uint32_t>(L.iv0),
                        ws->at<uint32_t>(L.ik1), ws->at<uint32_t>(L.iv1), ws->at<uint32_t>(L.hist),
                        ws->at<uint32_t>(L.scan32), &final1, s));
    ws->inst_keys = ws->at<uint32_t>(final1 ? L.ik1 : L.ik0);
    ws->inst_vals = ws->at<uint32_t>(final1 ? L.iv1 : L.iv0);
    uint2 *ranges = ws->at<uint2>(L.ranges);
    CK(cudaMemsetAsync(ranges, 0, (size_t)2 * ws->tiles * sizeof(uint2), s));
    CK(launch_ranges(ws->inst_keys, st, ws->caps.max_instances, 2 * (int64_t)ws->tiles, ranges, ws->sms, s));
    CK(launch_tile_order(ranges, ws->tiles, views, ws->V, ws->at<TileWorkDev>(L.work), ws->at<int32_t>(L.order),
                         ws->at<uint32_t>(L.vhist), ws->at<uint32_t>(L.voff), ws->at<uint32_t>(L.vt),
                         ws->at<uint32_t>(L.vbase), ws->at<uint32_t>(L.vscan), ws->sms, s));
    prof_end(ws, pk1, s);
    ws->stage = 2;
    return SDGR_OK;
}

static float exp2_cut(float K) { return -0.5f * LOG2E * K * K; }

// Schedule of raster kernel `kernel` (0 intensity, 1 splat, 2 splat adjoint,
// 3 intensity adjoint) under the workspace's schedule mode; a persistent
// launch gets its item counter zeroed first.
static cudaError_t raster_sched(sdgr_ws *ws, int kernel, cudaStream_t s, TileSched &sc) {
    const int plane = (kernel == 1 || kernel == 2) ? 1 : 0;
    sc.order = nullptr;
    sc.work = ws->at<TileWorkDev>(ws->L.work);
    sc.plane = plane;
    sc.slot = kernel;
    sc.persistent_grid = 0;
    sc.ntiles = ws->tiles;
    const int *sizes = nullptr;
    stage_batch_options(kernel, &sizes);
    sc.nb = ws->stage_batch[kernel] > 0 ? ws->stage_batch[kernel] : sizes[0];
    if (!(ws->sched & SDGR_SCHED_ORDERED)) return cudaSuccess;
    sc.order = ws->at<int32_t>(ws->L.order) + (size_t)plane * ws->tiles;
    if (ws->sched & SDGR_SCHED_PERSISTENT) {
        sc.persistent_grid = ws->sms * raster_blocks_per_sm(kernel, sc.nb);
        return cudaMemsetAsync(&sc.work->next[kernel], 0, sizeof(int32_t), s);
    }
    return cudaSuccess;
}

static float t_floor(float T_min) {
    const float f = 7.888609052210118e-31f;  // 2^-100
    return T_min > f ? T_min : f;
}

sdgr_status sdgr_render_fwd(sdgr_ws *ws, float *images, float *intensity, void *stream) {
    if (!ws) return SDGR_ERR_INVALID;
    if (ws->stage < 2) return SDGR_ERR_STATE;
    if (ws->npix > 0 && !images) return SDGR_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Layout &L = ws->L;
    const StatusDev *st = ws->at<StatusDev>(L.status);
    const ViewDev *views = ws->at<ViewDev>(L.views);
    const uint2 *ranges = ws->at<uint2>(L.ranges);
    const float cut = exp2_cut(ws->cfg.cutoff_K);
    float *A = ws->at<float>(L.A);
    if (ws->VG > 0) CK(cudaMemsetAsync(A, 0, (size_t)ws->VG * 4, s));
    // a work list skips tiles with empty lists: their pixels stay 0
    if ((ws->sched & SDGR_SCHED_ORDERED) && ws->npix > 0) CK(cudaMemsetAsync(images, 0, (size_t)ws->npix * 4, s));
    TileSched sc;
    CK(raster_sched(ws, 0, s, sc));
    int pk = prof_begin(ws, SDGR_STAGE_INTENSITY_FWD, s);
    CK(launch_intensity_fwd(ranges, ws->inst_vals, ws->at<CompRec>(L.comp), views, ws->V, ws->tiles, cut,
                            t_floor(ws->cfg.T_min), ws->cfg.alpha_mode, st, A, ws->at<float>(L.Tend),
                            ws->at<int32_t>(L.last), sc, s));
    prof_end(ws, pk, s);
    CK(raster_sched(ws, 1, s, sc));
    pk = prof_begin(ws, SDGR_STAGE_SPLAT_FWD, s);
    CK(launch_splat_fwd(ranges + ws->tiles, ws->inst_vals, ws->at<ImgRec>(L.img), ws->at<CompRec>(L.comp), A, views,
                        ws->V, ws->tiles, cut, st, images, sc, s));
    prof_end(ws, pk, s);
    if (intensity) CK(launch_intensity_out(ws->at<CompRec>(L.comp), A, ws->VG, intensity, ws->sms, s));
    ws->stage = 3;
    return SDGR_OK;
}

sdgr_status sdgr_render_bwd(sdgr_ws *ws, const float *dL_dimages, float *grads, int32_t accumulate, void *stream) {
    if (!ws) return SDGR_ERR_INVALID;
    if (ws->stage < 3) return SDGR_ERR_STATE;
    if ((ws->npix > 0 && !dL_dimages) || (ws->n_gauss > 0 && (!grads || ((uintptr_t)grads) % 16 != 0)))
        return SDGR_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Layout &L = ws->L;
    const StatusDev *st = ws->at<StatusDev>(L.status);
    const ViewDev *views = ws->at<ViewDev>(L.views);
    const uint2 *ranges = ws->at<uint2>(L.ranges);
    const float cut = exp2_cut(ws->cfg.cutoff_K);
    float4 *accI = ws->at<float4>(L.accI), *accC = ws->at<float4>(L.accC);
    if (ws->VG > 0) {
        CK(cudaMemsetAsync(accI, 0, (size_t)ws->VG * 2 * sizeof(float4), s));
        CK(cudaMemsetAsync(accC, 0, (size_t)ws->VG * 2 * sizeof(float4), s));
    }
    if (ws->n_gauss > 0 && !accumulate) CK(cudaMemsetAsync(grads, 0, (size_t)ws->n_gauss * 12 * 4, s));
    float *dsh = ws->sh ? ws->dsh : nullptr;
    if (dsh && ws->n_gauss > 0 && !accumulate) CK(cudaMemsetAsync(dsh, 0, (size_t)ws->n_gauss * 16 * 4, s));
    TileSched sc;
    CK(raster_sched(ws, 2, s, sc));
    int pk = prof_begin(ws, SDGR_STAGE_SPLAT_BWD, s);
    CK(launch_splat_bwd(ranges + ws->tiles, ws->inst_vals, ws->at<ImgRec>(L.img), dL_dimages, views, ws->V, ws->tiles,
                        cut, st, accI, sc, s));
    prof_end(ws, pk, s);
    CK(raster_sched(ws, 3, s, sc));
    pk = prof_begin(ws, SDGR_STAGE_INTENSITY_BWD, s);
    CK(launch_intensity_bwd(ranges, ws->inst_vals, ws->at<CompRec>(L.comp), ws->at<ImgRec>(L.img), accI,
                            ws->at<float>(L.Tend), ws->at<int32_t>(L.last), views, ws->V, ws->tiles, cut,
                            ws->cfg.alpha_mode, st, accC, sc, s));
    prof_end(ws, pk, s);
    pk = prof_begin(ws, SDGR_STAGE_PARAM_BWD, s);
    CK(launch_param_bwd(reinterpret_cast<const float4 *>(ws->params), views, ws->at<SceneDev>(L.scenes),
                        ws->at<int32_t>(L.scene_views), ws->n_scenes, ws->n_gauss, ws->cfg.dilation_eps,
                        ws->cfg.norm_mode, ws->cfg.alpha_mode, ws->at<float>(L.A), ws->at<CompRec>(L.comp), accI,
                        accC, st,
                        reinterpret_cast<float4 *>(grads),
                        reinterpret_cast<float4 *>(dsh), ws->dens_accum, ws->dens_count, ws->sms, s));
    prof_end(ws, pk, s);
    return SDGR_OK;
}

sdgr_status sdgr_set_schedule(sdgr_ws *ws, int32_t mode) {
    if (!ws || (mode & ~(SDGR_SCHED_ORDERED | SDGR_SCHED_PERSISTENT)) ||
        ((mode & SDGR_SCHED_PERSISTENT) && !(mode & SDGR_SCHED_ORDERED)))
        return SDGR_ERR_INVALID;
    ws->sched = mode;
    return SDGR_OK;
}

sdgr_status sdgr_device_selfcheck(uint32_t *flags, void *stream) {
    if (!flags || ((uintptr_t)flags) % 4 != 0) return SDGR_ERR_INVALID;
    return launch_selfcheck(flags, static_cast<cudaStream_t>(stream)) == cudaSuccess ? SDGR_OK : SDGR_ERR_CUDA;
}

sdgr_status sdgr_pipe_rates(void *scratch, double *rates, void *stream) {
    if (!scratch || !rates || ((uintptr_t)scratch) % 16 != 0) return SDGR_ERR_INVALID;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float *sink = static_cast<float *>(scratch);
    unsigned long long *cyc = reinterpret_cast<unsigned long long *>(static_cast<char *>(scratch) + 4096);
    static const int iters[SDGR_PIPE_RATE_KINDS] = {4096, 1024, 1024, 2048, 2048, 4096, 2048, 2048};
    for (int op = 0; op < SDGR_PIPE_RATE_KINDS; ++op) {
        CK(cudaMemsetAsync(cyc, 0, sizeof(*cyc), s));
        int bps = 0;
        CK(launch_pipe_rate(op, iters[op], sink, cyc, &bps, sms, s));
        CK(cudaStreamSynchronize(s));
        unsigned long long c = 0;
        CK(cudaMemcpy(&c, cyc, sizeof(c), cudaMemcpyDeviceToHost));
        // instructions counted per thread and iteration: 8, 9 for the rcp
        // stream (its rcp's fma included), 16 for the alternating streams
        const double per_iter = op == 4 ? 9.0 : (op >= 6 ? 16.0 : 8.0);
        rates[op] = c ? (double)bps * 1024.0 * iters[op] * per_iter / (double)c : 0.0;
    }
    return SDGR_OK;
}

int32_t sdgr_stage_batch_options(int32_t kernel, int32_t *sizes, int32_t max_sizes) {
    const int *opt = nullptr;
    const int n = stage_batch_options(kernel, &opt);
    for (int i = 0; i < n && i < max_sizes && sizes; ++i) sizes[i] = opt[i];
    return n;
}

sdgr_status sdgr_set_stage_batch(sdgr_ws *ws, int32_t kernel, int32_t records) {
    if (!ws || kernel < 0 || kernel > 3) return SDGR_ERR_INVALID;
    if (records == 0) {
        ws->stage_batch[kernel] = 0;
        return SDGR_OK;
    }
    const int *opt = nullptr;
    const int n = stage_batch_options(kernel, &opt);
    for (int i = 0; i < n; ++i)
        if (opt[i] == records) {
            ws->stage_batch[kernel] = records;
            return SDGR_OK;
        }
    return SDGR_ERR_INVALID;
}

sdgr_status sdgr_set_densify_stats(sdgr_ws *ws, float *accum, float *count) {
    if (!ws || ((accum == nullptr) != (count == nullptr))) return SDGR_ERR_INVALID;
    ws->dens_accum = accum;
    ws->dens_count = count;
    return SDGR_OK;
}

sdgr_status sdgr_set_sh(sdgr_ws *ws, const float *sh, float *dsh, int32_t degree) {
    if (!ws || degree < 0 || degree > 3) return SDGR_ERR_INVALID;
    if (((uintptr_t)sh | (uintptr_t)dsh) % 16 != 0) return SDGR_ERR_INVALID;
    ws->sh = sh;
    ws->dsh = dsh;
    ws->sh_degree = sh ? degree : 0;
    return SDGR_OK;
}

sdgr_status sdgr_adam_step(float *params, const float *grads, float *m, float *v, int64_t N, const float *lr,
                           float b1, float b2, float eps, int32_t step, void *stream) {
    if (N < 0 || step < 1 || !lr) return SDGR_ERR_INVALID;
    if (N == 0) return SDGR_OK;
    if (!params || !grads || !m || !v) return SDGR_ERR_INVALID;
    if (((uintptr_t)params | (uintptr_t)grads | (uintptr_t)m | (uintptr_t)v) % 16 != 0) return SDGR_ERR_INVALID;
    if (!(b1 >= 0.f && b1 < 1.f && b2 >= 0.f && b2 < 1.f && eps >= 0.f)) return SDGR_ERR_INVALID;
    int dev = 0, sms = 148;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(launch_adam(reinterpret_cast<float4 *>(params), reinterpret_cast<const float4 *>(grads),
                   reinterpret_cast<float4 *>(m), reinterpret_cast<float4 *>(v), N * 3, lr, b1, b2, eps, step, sms,
                   static_cast<cudaStream_t>(stream)));
    return SDGR_OK;
}

sdgr_status sdgr_adam_step_flat(float *x, const float *grads, float *m, float *v, int64_t n, float lr, float b1,
                                float b2, float eps, int32_t step, void *stream) {
    if (n < 0 || n % 4 != 0 || step < 1) return SDGR_ERR_INVALID;
    if (n == 0) return SDGR_OK;
    if (!x || !grads || !m || !v) return SDGR_ERR_INVALID;
    if (((uintptr_t)x | (uintptr_t)grads | (uintptr_t)m | (uintptr_t)v) % 16 != 0) return SDGR_ERR_INVALID;
    if (!(b1 >= 0.f && b1 < 1.f && b2 >= 0.f && b2 < 1.f && eps >= 0.f)) return SDGR_ERR_INVALID;
    int dev = 0, sms = 148;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const float lr5[5] = {lr, lr, lr, lr, lr};  // one rate for every component
    CK(launch_adam(reinterpret_cast<float4 *>(x), reinterpret_cast<const float4 *>(grads),
                   reinterpret_cast<float4 *>(m), reinterpret_cast<float4 *>(v), n / 4, lr5, b1, b2, eps, step, sms,
                   static_cast<cudaStream_t>(stream)));
    return SDGR_OK;
}

sdgr_status sdgr_adam_step_device(float *params, const float *grads, float *m, float *v, int64_t N, const float *lr,
                                  float b1, float b2, float eps, int32_t *step, void *stream) {
    if (N < 0 || !lr || !step) return SDGR_ERR_INVALID;
    if (N > 0 && (!params || !grads || !m || !v)) return SDGR_ERR_INVALID;
    if (((uintptr_t)params | (uintptr_t)grads | (uintptr_t)m | (uintptr_t)v) % 16 != 0) return SDGR_ERR_INVALID;
    if (!(b1 >= 0.f && b1 < 1.f && b2 >= 0.f && b2 < 1.f && eps >= 0.f)) return SDGR_ERR_INVALID;
    int dev = 0, sms = 148;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(launch_adam_dev(reinterpret_cast<float4 *>(params), reinterpret_cast<const float4 *>(grads),
                       reinterpret_cast<float4 *>(m), reinterpret_cast<float4 *>(v), N * 3, lr, b1, b2, eps, step, sms,
                       static_cast<cudaStream_t>(stream)));
    return SDGR_OK;
}

sdgr_status sdgr_l1_loss(const float *images, const float *targets, int64_t npix, float *dL_dimages, float *loss,
                         void *stream) {
    if (npix < 0 || !loss || (npix > 0 && (!images || !targets || !dL_dimages))) return SDGR_ERR_INVALID;
    int dev = 0, sms = 148;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(launch_l1(images, targets, npix, dL_dimages, loss, sms, static_cast<cudaStream_t>(stream)));
    return SDGR_OK;
}

sdgr_status sdgr_count_pairs(sdgr_ws *ws, int64_t *pairs, void *stream) {
    if (!ws || !pairs) return SDGR_ERR_INVALID;
    if (ws->stage < 2) return SDGR_ERR_STATE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    StatusDev *st = ws->at<StatusDev>(ws->L.status);
    CK(cudaMemsetAsync(st->pairs, 0, sizeof(st->pairs), s));
    CK(launch_count_pairs(ws->at<uint2>(ws->L.ranges), ws->inst_vals, ws->at<CompRec>(ws->L.comp),
                          ws->at<ImgRec>(ws->L.img), ws->at<ViewDev>(ws->L.views), ws->V, ws->tiles,
                          exp2_cut(ws->cfg.cutoff_K), st, s));
    CK(cudaStreamSynchronize(s));
    unsigned long long h[2];
    CK(cudaMemcpy(h, st->pairs, sizeof(h), cudaMemcpyDeviceToHost));
    pairs[0] = (int64_t)h[0];
    pairs[1] = (int64_t)h[1];
    return SDGR_OK;
}

int64_t sdgr_launch_count(void) { return (int64_t)g_launches.load(); }

sdgr_status sdgr_profile_enable(sdgr_ws *ws, int32_t enable) {
    if (!ws) return SDGR_ERR_INVALID;
    if (enable && ws->prof_ev.empty()) {
        ws->prof_ev.assign(2 * PROF_PAIRS, nullptr);
        ws->prof_stage.assign(PROF_PAIRS, 0);
        for (auto &e : ws->prof_ev) CK(cudaEventCreate(&e));
    }
    ws->prof_on = enable != 0;
    return SDGR_OK;
}

sdgr_status sdgr_profile_read(sdgr_ws *ws, double *ms, int64_t *launches, int32_t reset) {
    if (!ws || !ms || !launches) return SDGR_ERR_INVALID;
    CK(prof_harvest(ws));
    for (int k = 0; k < SDGR_NUM_STAGES; ++k) {
        ms[k] = ws->prof_ms[k];
        launches[k] = ws->prof_n[k];
        if (reset) {
            ws->prof_ms[k] = 0.0;
            ws->prof_n[k] = 0;
        }
    }
    return SDGR_OK;
}

sdgr_status sdgr_copy_status_async(sdgr_ws *ws, void *host_dst, void *stream) {
    if (!ws || !host_dst) return SDGR_ERR_INVALID;
    CK(cudaMemcpyAsync(host_dst, ws->base + ws->L.status, 16, cudaMemcpyDeviceToHost,
                       static_cast<cudaStream_t>(stream)));
    return SDGR_OK;
}

sdgr_status sdgr_read_status(sdgr_ws *ws, int64_t *required_instances) {
    if (!ws) return SDGR_ERR_INVALID;
    StatusDev h;
    CK(cudaMemcpy(&h, ws->base + ws->L.status, sizeof(h), cudaMemcpyDeviceToHost));
    if (required_instances) *required_instances = h.required;
    return (sdgr_status)h.code;
}

}  // extern "C"
