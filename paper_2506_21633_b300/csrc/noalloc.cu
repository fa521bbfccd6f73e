// noalloc.cu -- forward render whose workspace is a fixed device array owned
// by the library, for callers that cannot allocate device memory themselves.
// It drives the same public calls as any other caller (sdgr_preprocess,
// sdgr_bin_sort, sdgr_render_fwd); only the workspace buffer differs.
#include <string.h>

#include <mutex>

#include "sdgr_internal.cuh"

namespace {

// The scratch.  In host code this name is only a stand-in for the device
// array: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SDGR_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
constexpr int64_t MAX_TILES = 16384;

struct DeviceState {
    bool ready = false;
    void *scratch = nullptr;  // device address of g_noalloc_scratch on this device
    sdgr_caps caps;           // capacities the scratch holds
    sdgr_ws *ws = nullptr;    // host handle bound to the scratch (rebuilt when cfg changes)
    sdgr_cfg cfg;
};

std::mutex g_lock;
DeviceState g_dev[MAX_DEVICES];

// Largest instance capacity whose workspace fits the scratch.
bool fit_caps(const sdgr_cfg *cfg, sdgr_caps *caps) {
    caps->max_views = SDGR_NOALLOC_MAX_VIEWS;
    caps->max_scenes = 1;
    caps->max_gaussians = SDGR_NOALLOC_MAX_GAUSSIANS;
    caps->max_view_gauss = (int64_t)SDGR_NOALLOC_MAX_GAUSSIANS * SDGR_NOALLOC_MAX_VIEWS;
    caps->max_pixels = SDGR_NOALLOC_MAX_PIXELS;
    caps->max_tiles = MAX_TILES;
    int64_t lo = 0, hi = (int64_t)SDGR_NOALLOC_SCRATCH_BYTES / 8;
    caps->max_instances = 0;
    size_t bytes = 0;
    if (sdgr_workspace_size(cfg, caps, &bytes) != SDGR_OK || bytes > SDGR_NOALLOC_SCRATCH_BYTES) return false;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        caps->max_instances = mid;
        if (sdgr_workspace_size(cfg, caps, &bytes) == SDGR_OK && bytes <= SDGR_NOALLOC_SCRATCH_BYTES) lo = mid;
        else hi = mid - 1;
    }
    caps->max_instances = lo;
    return lo > 0;
}

}  // namespace

extern "C" sdgr_status sdgr_render_fwd_noalloc(const float *params, int64_t N, const sdgr_view *views, int32_t V,
                                               const sdgr_cfg *cfg, float *images, float *intensity, void *stream) {
    if (!cfg || !views || !images || V < 1 || V > SDGR_NOALLOC_MAX_VIEWS || N < 0 ||
        N > SDGR_NOALLOC_MAX_GAUSSIANS)
        return SDGR_ERR_INVALID;
    if (N > 0 && (!params || ((uintptr_t)params) % 16 != 0)) return SDGR_ERR_INVALID;
    const int64_t offsets[2] = {0, N};
    sdgr_caps need;
    if (sdgr_caps_for(views, V, offsets, 1, 0, &need) != SDGR_OK) return SDGR_ERR_INVALID;
    if (need.max_pixels > SDGR_NOALLOC_MAX_PIXELS || need.max_tiles > MAX_TILES) return SDGR_ERR_INVALID;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return SDGR_ERR_CUDA;
    std::lock_guard<std::mutex> guard(g_lock);
    DeviceState &d = g_dev[dev];
    if (!d.ready) {
        // once per device, with that device current
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return SDGR_ERR_CUDA;
        d.scratch = ptr;
        d.ready = true;
    }
    if (!d.ws || memcmp(&d.cfg, cfg, sizeof(sdgr_cfg)) != 0) {
        if (d.ws) {
            sdgr_ws_destroy(d.ws);
            d.ws = nullptr;
        }
        if (!fit_caps(cfg, &d.caps)) return SDGR_ERR_INVALID;
        sdgr_status st = sdgr_ws_create(&d.ws, d.scratch, SDGR_NOALLOC_SCRATCH_BYTES, cfg, &d.caps);
        if (st != SDGR_OK) {
            d.ws = nullptr;
            return st;
        }
        d.cfg = *cfg;
    }
    sdgr_status st = sdgr_preprocess(d.ws, params, offsets, 1, views, V, stream);
    if (st == SDGR_OK) st = sdgr_bin_sort(d.ws, stream);
    if (st == SDGR_OK) st = sdgr_render_fwd(d.ws, images, intensity, stream);
    if (st != SDGR_OK) return st;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return SDGR_ERR_CUDA;
    return sdgr_read_status(d.ws, nullptr);
}
