// common.cu -- error reporting, device queries and grid geometry for the C ABI.
#include <cstdarg>
#include <cstring>

#include "nacc_internal.cuh"

namespace nacc {

namespace {
thread_local char g_err[512] = "";
int g_sm_count[64] = {0};
}  // namespace

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = '\0'; }

thread_local cudaEvent_t g_count_ev[2] = {nullptr, nullptr};

cudaEvent_t* march_count_events() { return g_count_ev; }

int sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev >= 0 && dev < 64 && g_sm_count[dev] > 0) return g_sm_count[dev];
    int n = 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    if (dev >= 0 && dev < 64) g_sm_count[dev] = n;
    return n;
}

// Level l: cen = (min+max)*0.5, half = (max-min)*0.5, lmin = cen - half*2^l,
// lmax = cen + half*2^l, scale = res/(lmax-lmin), width = (lmax-lmin)/res,
// every operation an individually rounded FP32 operation (the host code is
// compiled with -ffp-contract=off).
bool make_geom(const nacc_grid* grid, GridGeom* g, bool need_bits) {
    if (!grid) {
        set_error("grid is NULL");
        return false;
    }
    if (grid->n_levels < 1 || grid->n_levels > NACC_MAX_LEVELS) {
        set_error("grid n_levels=%d outside [1, %d]", grid->n_levels, NACC_MAX_LEVELS);
        return false;
    }
    if (grid->res < 1 || grid->res > 1024) {
        set_error("grid res=%d outside [1, 1024]", grid->res);
        return false;
    }
    int64_t r3 = (int64_t)grid->res * grid->res * grid->res;
    if (r3 % 32 != 0) {
        set_error("grid res^3 = %lld is not a multiple of 32", (long long)r3);
        return false;
    }
    if (need_bits && !grid->bits) {
        set_error("grid bits is NULL");
        return false;
    }
    for (int a = 0; a < 3; ++a) {
        if (!(grid->aabb_min[a] < grid->aabb_max[a]) || !std::isfinite(grid->aabb_min[a]) ||
            !std::isfinite(grid->aabb_max[a])) {
            set_error("grid aabb axis %d: need finite min < max", a);
            return false;
        }
    }
    std::memset(g, 0, sizeof(*g));
    for (int l = 0; l < grid->n_levels; ++l) {
        volatile float f = (float)(1 << l);
        for (int a = 0; a < 3; ++a) {
            volatile float cen = (grid->aabb_min[a] + grid->aabb_max[a]) * 0.5f;
            volatile float half = (grid->aabb_max[a] - grid->aabb_min[a]) * 0.5f;
            volatile float hs = half * f;
            volatile float lo = cen - hs;
            volatile float hi = cen + hs;
            volatile float ext = hi - lo;
            g->lv[l].lmin[a] = lo;
            g->lv[l].lmax[a] = hi;
            g->lv[l].scale[a] = (float)grid->res / ext;
            g->lv[l].width[a] = ext / (float)grid->res;
            if (!std::isfinite(lo) || !std::isfinite(hi) || !(ext > 0.0f)) {
                set_error("grid level %d box is not finite", l);
                return false;
            }
        }
    }
    g->res = grid->res;
    g->n_levels = grid->n_levels;
    g->bits = grid->bits;
    return true;
}

}  // namespace nacc

extern "C" const char* nacc_last_error(void) { return nacc::g_err; }

extern "C" int nacc_version(void) { return 100; }
