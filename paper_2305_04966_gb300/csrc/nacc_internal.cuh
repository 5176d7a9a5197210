// nacc_internal.cuh -- shared helpers of the CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>

#include "../../include/nacc.h"
#include "../../include/nacc_harness.h"
#include "../../include/nacc_proposal.h"

namespace nacc {

// ---------------------------------------------------------------------------
// error reporting (thread-local message, no exceptions across the ABI)
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();
int sm_count();  // multiprocessors of the current device (cached per device)
// Caller-owned events that the marches record around their count phase on
// the calling host thread (diagnostics; both null when off).
cudaEvent_t* march_count_events();
unsigned int mlp_take_status();  // reads and clears the proposal network's device status word

#define NACC_CHECK_ARG(cond, ...)                      \
    do {                                               \
        if (!(cond)) {                                 \
            ::nacc::set_error(__VA_ARGS__);            \
            return NACC_ERR_INVALID_ARG;               \
        }                                              \
    } while (0)

#define NACC_CUDA_TRY(expr)                                                              \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            ::nacc::set_error("%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                              __LINE__);                                                 \
            return NACC_ERR_CUDA;                                                        \
        }                                                                                \
    } while (0)

// Check the launch that was just enqueued.
#define NACC_LAUNCH_CHECK() NACC_CUDA_TRY(cudaGetLastError())

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ---------------------------------------------------------------------------
// grid geometry, computed once on the host in FP32 (see nacc_grid)
// ---------------------------------------------------------------------------
struct Level {
    float lmin[3], lmax[3], scale[3], width[3];
};

struct GridGeom {
    Level lv[NACC_MAX_LEVELS];
    int res;
    int n_levels;
    const uint32_t* bits;
};

// Fills `g` from `grid`; returns false (with the error set) on bad arguments.
bool make_geom(const nacc_grid* grid, GridGeom* g, bool need_bits);

// Early-stop optical-depth threshold: T < eps <=> depth > -ln(eps).
inline float tau_threshold(float eps) {
    if (!(eps > 0.0f)) return INFINITY;
    return (float)(-std::log((double)eps));
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------

// SplitMix64 output number counter+1 of the stream seeded with `seed`
// (Steele, Lea, Flood 2014), used as a counter-based generator.
__host__ __device__ inline uint64_t splitmix64(uint64_t seed, uint64_t counter) {
    uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ inline float u01_from_bits(uint64_t h) {
    return (float)(h >> 40) * 5.9604644775390625e-8f;  // 2^-24
}

// Blob parameters staged in shared memory: centre, coefficient -0.5/std^2
// (computed as fl(-0.5 / fl(std*std))), peak, colour.
struct BlobS {
    float mx, my, mz, coef, peak, r, g, b;
};

// Loads up to n blobs into shared memory (call by the whole block, then sync).
__device__ inline void stage_blobs(BlobS* s, const nacc_blob_field& f, bool with_rgb) {
    for (int b = threadIdx.x; b < f.n_blobs; b += blockDim.x) {
        BlobS v;
        v.mx = f.mu[3 * b + 0];
        v.my = f.mu[3 * b + 1];
        v.mz = f.mu[3 * b + 2];
        float sd = f.std[b];
        float sd2 = __fmul_rn(sd, sd);
        v.coef = __fdiv_rn(-0.5f, sd2);
        v.peak = f.peak[b];
        if (with_rgb) {
            v.r = f.rgb[3 * b + 0];
            v.g = f.rgb[3 * b + 1];
            v.b = f.rgb[3 * b + 2];
        } else {
            v.r = v.g = v.b = 0.0f;
        }
        s[b] = v;
    }
}

// FP32 blob density with a fixed, individually rounded operation order:
//   r2 = (dx*dx + dy*dy) + dz*dz; s += peak * expf(r2 * coef).
__device__ __forceinline__ float blob_sigma(const BlobS* s, int n, float x, float y, float z) {
    float acc = 0.0f;
    for (int b = 0; b < n; ++b) {
        const BlobS& v = s[b];
        float dx = __fsub_rn(x, v.mx);
        float dy = __fsub_rn(y, v.my);
        float dz = __fsub_rn(z, v.mz);
        float r2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
        r2 = __fadd_rn(r2, __fmul_rn(dz, dz));
        float e = expf(__fmul_rn(r2, v.coef));
        acc = __fadd_rn(acc, __fmul_rn(v.peak, e));
    }
    return acc;
}

constexpr int kMaxBlobs = 1024;

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

}  // namespace nacc
