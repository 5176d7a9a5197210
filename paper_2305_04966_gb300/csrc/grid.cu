// grid.cu -- estimator update (nacc_grid_points, nacc_update_grid).
//
// Eq. 4 (the update F: T^{k-1} -> T^k) in the EMA form of Sec. 3.1
// "Spatial Skipping", and the binarisation 1[sigma > tau] of Table 1.
// Three kernels: EMA + per-block FP64 partial sums, a one-block reduction to
// the FP64 mean and threshold, and a warp-ballot bit packer (32 cells = one
// word per warp).  No atomics: the mean is deterministic.
#include <cuda.h>

#include <mutex>

#include "nacc_internal.cuh"

namespace nacc {
namespace {

constexpr int kEmaThreads = 256;
constexpr int kEmaItems = 8;  // cells per thread
constexpr int kEmaCells = kEmaThreads * kEmaItems;

template <typename I>  // index type: uint32_t when every cell index fits, else int64_t
__global__ void __launch_bounds__(256)
    k_grid_points(GridGeom g, uint64_t key, int jitter, int64_t n_cells, float* __restrict__ xyz) {
    const I res = (I)g.res, r2 = res * res, r3 = r2 * res;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cells;
         c += (int64_t)gridDim.x * blockDim.x) {
        const I ci = (I)c;
        const int l = (int)(ci / r3);
        const I w = ci - (I)l * r3;
        const I x = w / r2, yz = w - x * r2, y = yz / res;
        const int64_t i[3] = {(int64_t)x, (int64_t)y, (int64_t)(yz - y * res)};
        const Level& lv = g.lv[l];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float u = jitter ? u01_from_bits(splitmix64(key, (uint64_t)(3 * c + a))) : 0.5f;
            float q = __fadd_rn((float)i[a], u);
            xyz[3 * c + a] = __fadd_rn(lv.lmin[a], __fmul_rn(q, lv.width[a]));
        }
    }
}

__global__ void __launch_bounds__(kEmaThreads)
    k_ema(float* __restrict__ ema, const float* __restrict__ dens, float decay, float omd,
          int64_t n, double* __restrict__ partial, int n_frames) {
    const int64_t base = (int64_t)blockIdx.x * kEmaCells;
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < kEmaItems; ++j) {
        int64_t c = base + j * kEmaThreads + threadIdx.x;
        if (c < n) {
            float dc = __ldcs(dens + c);
            for (int f = 1; f < n_frames; ++f) dc = fmaxf(dc, __ldcs(dens + (int64_t)f * n + c));
            float a = __fmul_rn(decay, ema[c]);
            float b = __fmul_rn(omd, dc);
            float e = __fadd_rn(a, b);
            ema[c] = e;
            acc += (double)e;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double s_w[kEmaThreads / 32];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kEmaThreads / 32; ++w) t += s_w[w];
        partial[blockIdx.x] = t;
    }
}

// The same EMA with 128-bit accesses (ema, dens 16-byte aligned; n a
// multiple of 4): thread t of block b owns the float4 groups
// b*kEmaCells/4 + j*kEmaThreads + t, j < kEmaItems/4 -- the same cells per
// block, so the per-block partial sums cover the same cells.
// n_frames > 1 (dynamic scenes): the density fed to the EMA is the maximum
// over the frames dens[f * n + c] (the grid marks the maximum occupancy over
// all timestamps).
__global__ void __launch_bounds__(kEmaThreads)
    k_ema4(float* __restrict__ ema, const float* __restrict__ dens, float decay, float omd, int64_t n,
           double* __restrict__ partial, int n_frames) {
    const int64_t base = (int64_t)blockIdx.x * (kEmaCells / 4);
    const int64_t n4 = n / 4;
    float4* e4 = reinterpret_cast<float4*>(ema);
    const float4* d4 = reinterpret_cast<const float4*>(dens);
    float4 ev[kEmaItems / 4], dv[kEmaItems / 4];
#pragma unroll
    for (int j = 0; j < kEmaItems / 4; ++j) {
        const int64_t q = base + j * kEmaThreads + threadIdx.x;
        if (q < n4) {
            ev[j] = e4[q];
            dv[j] = __ldcs(d4 + q);
            for (int f = 1; f < n_frames; ++f) {
                const float4 u = __ldcs(d4 + (int64_t)f * n4 + q);
                dv[j].x = fmaxf(dv[j].x, u.x);
                dv[j].y = fmaxf(dv[j].y, u.y);
                dv[j].z = fmaxf(dv[j].z, u.z);
                dv[j].w = fmaxf(dv[j].w, u.w);
            }
        }
    }
    // the thread's 8 cells summed in FP32 with Neumaier's compensation, then
    // converted to FP64 once (error ~n u^2 of the sum: FP64-grade without a
    // slow FP64 conversion and add per cell)
    float sh = 0.0f, sc = 0.0f;
    auto add = [&](float v) {
        const float t = sh + v;
        sc += fabsf(sh) >= fabsf(v) ? (sh - t) + v : (v - t) + sh;
        sh = t;
    };
#pragma unroll
    for (int j = 0; j < kEmaItems / 4; ++j) {
        const int64_t q = base + j * kEmaThreads + threadIdx.x;
        if (q < n4) {
            float4 r;
            r.x = __fadd_rn(__fmul_rn(decay, ev[j].x), __fmul_rn(omd, dv[j].x));
            r.y = __fadd_rn(__fmul_rn(decay, ev[j].y), __fmul_rn(omd, dv[j].y));
            r.z = __fadd_rn(__fmul_rn(decay, ev[j].z), __fmul_rn(omd, dv[j].z));
            r.w = __fadd_rn(__fmul_rn(decay, ev[j].w), __fmul_rn(omd, dv[j].w));
            e4[q] = r;
            add(r.x);
            add(r.y);
            add(r.z);
            add(r.w);
        }
    }
    double acc = (double)sh + (double)sc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double s_w[kEmaThreads / 32];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < kEmaThreads / 32; ++w) t += s_w[w];
        partial[blockIdx.x] = t;
    }
}

// One block: mean = sum(partial) / n; thr = max(thresh_abs, thresh_frac*mean).
__global__ void __launch_bounds__(1024)
    k_mean_thr(const double* __restrict__ partial, int64_t nb, int64_t n, double thresh_frac,
               double thresh_abs, double* __restrict__ out) {
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < nb; i += 1024) acc += partial[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double s_w[32];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 32; ++w) t += s_w[w];
        double mean = n > 0 ? t / (double)n : 0.0;
        double thr = thresh_frac * mean;
        if (thresh_abs > thr) thr = thresh_abs;
        // largest float <= thr: for a float e, (double)e > thr <=> e > thr32
        float thr32 = (float)thr;
        if ((double)thr32 > thr) thr32 = nextafterf(thr32, -INFINITY);
        out[0] = mean;
        out[1] = thr;
        out[2] = (double)thr32;
    }
}

__global__ void __launch_bounds__(256)
    k_pack_bits(const float* __restrict__ ema, int64_t n, const double* __restrict__ mt,
                uint32_t* __restrict__ bits) {
    const float thr = (float)mt[2];
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
         c += (int64_t)gridDim.x * blockDim.x) {
        bool occ = ema[c] > thr;
        unsigned m = __ballot_sync(0xffffffffu, occ);
        if ((threadIdx.x & 31) == 0) bits[c >> 5] = m;
    }
}

// The same packing with each thread building its own word from 32
// consecutive cells read as eight float4 (ema 16-byte aligned, n a multiple
// of 32).
__global__ void __launch_bounds__(256)
    k_pack_bits4(const float* __restrict__ ema, int64_t n, const double* __restrict__ mt,
                 uint32_t* __restrict__ bits) {
    const float thr = (float)mt[2];
    const int64_t words = n / 32;
    const float4* e4 = reinterpret_cast<const float4*>(ema);
    for (int64_t wd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; wd < words;
         wd += (int64_t)gridDim.x * blockDim.x) {
        float4 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = __ldcs(e4 + 8 * wd + j);
        uint32_t m = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            m |= (v[j].x > thr ? 1u : 0u) << (4 * j);
            m |= (v[j].y > thr ? 1u : 0u) << (4 * j + 1);
            m |= (v[j].z > thr ? 1u : 0u) << (4 * j + 2);
            m |= (v[j].w > thr ? 1u : 0u) << (4 * j + 3);
        }
        bits[wd] = m;
    }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// EMA -> mean and threshold -> bits, on caller scratch or the library's own.
int launch_update(float* ema, const float* density, float decay, int64_t n, double thresh_frac,
                  double thresh_abs, uint32_t* bits_out, double* partial, double* mt, cudaStream_t st,
                  int n_frames = 1) {
    const int64_t nb = (n + kEmaCells - 1) / kEmaCells;
    volatile float omd = 1.0f - decay;
    const bool vec = aligned16(ema) && aligned16(density) && n % 4 == 0;
    if (vec)
        k_ema4<<<(unsigned)nb, kEmaThreads, 0, st>>>(ema, density, decay, omd, n, partial, n_frames);
    else
        k_ema<<<(unsigned)nb, kEmaThreads, 0, st>>>(ema, density, decay, omd, n, partial, n_frames);
    NACC_LAUNCH_CHECK();
    k_mean_thr<<<1, 1024, 0, st>>>(partial, nb, n, thresh_frac, thresh_abs, mt);
    NACC_LAUNCH_CHECK();
    if (aligned16(ema)) {
        const int64_t words = n / 32;
        const int blocks = (int)std::min<int64_t>((words + 255) / 256, (int64_t)sm_count() * 8);
        k_pack_bits4<<<blocks, 256, 0, st>>>(ema, n, mt, bits_out);
    } else {
        const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 16);
        k_pack_bits<<<blocks, 256, 0, st>>>(ema, n, mt, bits_out);
    }
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}

// Cell of a packed sample's midpoint, the lattice march's FP32 definition:
// tm = (t0 + t1) * 0.5, x = o + d * tm, level = finest level whose box holds
// x, cell = clamp(floor((x - lmin) * scale)); flat index
// l*res^3 + (x*res + y)*res + z, or -1 outside every level.
__device__ __forceinline__ int64_t sample_cell(const GridGeom& g, const float* __restrict__ o,
                                               const float* __restrict__ d, int64_t r, float t0, float t1) {
    const float tm = __fmul_rn(__fadd_rn(t0, t1), 0.5f);
    float x[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = __fadd_rn(o[3 * r + a], __fmul_rn(d[3 * r + a], tm));
    int l = 0;
    for (; l < g.n_levels; ++l) {
        const Level& lv = g.lv[l];
        if (x[0] >= lv.lmin[0] && x[0] <= lv.lmax[0] && x[1] >= lv.lmin[1] && x[1] <= lv.lmax[1] &&
            x[2] >= lv.lmin[2] && x[2] <= lv.lmax[2])
            break;
    }
    if (l == g.n_levels) return -1;
    const Level& lv = g.lv[l];
    int64_t ic[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int c = (int)floorf(__fmul_rn(__fsub_rn(x[a], lv.lmin[a]), lv.scale[a]));
        ic[a] = c < 0 ? 0 : (c > g.res - 1 ? g.res - 1 : c);
    }
    const int64_t res = g.res;
    return (int64_t)l * res * res * res + (ic[0] * res + ic[1]) * res + ic[2];
}

// SGD-updated grid (the estimator's density updated by gradient descent
// through the rendering loss): density of each sample's cell, and the
// adjoint: the sample's dL/dsigma added into its cell.
template <bool kBackward>
__global__ void __launch_bounds__(256)
    k_grid_samples(GridGeom g, const float* __restrict__ o, const float* __restrict__ d,
                   const int32_t* __restrict__ ri, const float* __restrict__ t0, const float* __restrict__ t1,
                   const int64_t* __restrict__ n_samples, const float* __restrict__ dens_or_gsig,
                   float* __restrict__ out) {
    const int64_t S = *n_samples;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = sample_cell(g, o, d, ri[i], t0[i], t1[i]);
        if (kBackward) {
            if (c >= 0) atomicAdd(out + c, dens_or_gsig[i]);
        } else {
            out[i] = c >= 0 ? dens_or_gsig[c] : 0.0f;
        }
    }
}

// density = max(density - lr * grad, 0), grad = 0, bits = density > thresh.
__global__ void __launch_bounds__(256) k_grid_sgd(float* __restrict__ dens, float* __restrict__ grad, int64_t n,
                                                  float lr, float thresh, uint32_t* __restrict__ bits) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const float v = fmaxf(__fsub_rn(dens[c], __fmul_rn(lr, grad[c])), 0.0f);
        dens[c] = v;
        grad[c] = 0.0f;
        const unsigned m = __ballot_sync(0xffffffffu, v > thresh);
        if ((threadIdx.x & 31) == 0) bits[c >> 5] = m;
    }
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace nacc

using namespace nacc;

extern "C" int nacc_grid_points(const nacc_grid* grid, uint64_t seed, int64_t step, int32_t jitter,
                                float* xyz_out, void* stream) {
    clear_error();
    GridGeom g;
    if (!make_geom(grid, &g, false)) return NACC_ERR_INVALID_ARG;
    NACC_CHECK_ARG(xyz_out != nullptr, "xyz_out is NULL");
    const int64_t n = (int64_t)g.n_levels * g.res * g.res * g.res;
    const uint64_t key = seed ^ ((uint64_t)step << 32);
    int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 16);
    if (n <= (int64_t)0xffffffffll)
        k_grid_points<uint32_t><<<blocks, 256, 0, as_stream(stream)>>>(g, key, jitter ? 1 : 0, n, xyz_out);
    else
        k_grid_points<int64_t><<<blocks, 256, 0, as_stream(stream)>>>(g, key, jitter ? 1 : 0, n, xyz_out);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}

extern "C" size_t nacc_update_grid_scratch_bytes(int64_t n_cells) {
    if (n_cells < 0) return 0;
    int64_t nb = (n_cells + kEmaCells - 1) / kEmaCells;
    return align256(sizeof(double) * (size_t)(nb > 0 ? nb : 1)) + align256(3 * sizeof(double));
}

extern "C" int nacc_update_grid(const nacc_grid* grid, float* ema, const float* density,
                                float decay, float thresh_frac, float thresh_abs,
                                uint32_t* bits_out, void* scratch, size_t scratch_bytes,
                                void* stream) {
    clear_error();
    GridGeom g;
    if (!make_geom(grid, &g, false)) return NACC_ERR_INVALID_ARG;
    NACC_CHECK_ARG(ema && density && bits_out, "ema / density / bits_out is NULL");
    NACC_CHECK_ARG(decay >= 0.0f && decay <= 1.0f, "decay=%g outside [0, 1]", (double)decay);
    NACC_CHECK_ARG(std::isfinite(thresh_frac) && std::isfinite(thresh_abs), "thresholds must be finite");
    const int64_t n = (int64_t)g.n_levels * g.res * g.res * g.res;
    size_t need = nacc_update_grid_scratch_bytes(n);
    NACC_CHECK_ARG(scratch != nullptr && scratch_bytes >= need, "scratch too small: %zu < %zu bytes",
                   scratch_bytes, need);
    NACC_CHECK_ARG((reinterpret_cast<uintptr_t>(scratch) & 255) == 0, "scratch not 256-byte aligned");
    const int64_t nb = (n + kEmaCells - 1) / kEmaCells;
    double* partial = static_cast<double*>(scratch);
    double* mt = reinterpret_cast<double*>(static_cast<char*>(scratch) + align256(sizeof(double) * (size_t)nb));
    return launch_update(ema, density, decay, n, (double)thresh_frac, (double)thresh_abs, bits_out, partial, mt,
                         as_stream(stream));
}

// ---------------------------------------------------------------------------
// nacc_update_grid_noalloc: the same update with library-owned scratch.
//
// For callers that cannot call cudaMalloc (or any allocator) on the path that
// refreshes the grid -- for example code embedded in a host application that
// owns the whole device memory budget and forbids device allocations after
// start-up, or a latency-critical thread that must not pay for the implicit
// synchronisation an allocation can cause.  The FP64 partial sums and the
// (mean, threshold) pair live in one file-scope device array instead of a
// caller buffer.  Every GPU that loads this library holds the array until
// the process exits.
// ---------------------------------------------------------------------------

namespace nacc {
namespace {
constexpr int64_t kNoAllocMaxCells = int64_t(1) << 27;             // 134,217,728 cells
constexpr int64_t kNoAllocMaxBlocks = kNoAllocMaxCells / kEmaCells;  // 65,536 partial sums
}  // namespace
}  // namespace nacc

// 65,536 FP64 partial sums + mean + threshold (FP64 and FP32): 512 KiB + 24 B per device.
static __device__ __align__(256) double nacc_update_noalloc_scratch[nacc::kNoAllocMaxBlocks + 3];

namespace nacc {
namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
struct NoAllocEntry {
    unsigned long long ctx_id;  // unique per context for the life of the process (never reused)
    double* ptr;
};
NoAllocEntry g_noalloc[kNoAllocMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Unique id of the current context (0 if the driver cannot say).  The two
// driver calls are resolved through the runtime, so the library does not
// link the driver library itself.
unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the array in the current context (the host-side name of
// a __device__ variable is not a device address).  Cached per device together
// with the id of the context it was taken in, and looked up again when that
// context changes: after a device reset, or when the primary context is torn
// down and created again, the module (and the array) can load at another
// address.  Without a context id every call looks the address up.
int noalloc_scratch(double** out) {
    int dev = 0;
    NACC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("device %d is beyond the %d devices this entry point supports", dev, kNoAllocMaxDevices);
        return NACC_ERR_UNSUPPORTED;
    }
    const unsigned long long id = current_ctx_id();
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (id == 0 || g_noalloc[dev].ctx_id != id || !g_noalloc[dev].ptr) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, nacc_update_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_error("cudaGetSymbolAddress(nacc_update_noalloc_scratch) failed on device %d: %s", dev,
                      cudaGetErrorString(e));
            return NACC_ERR_CUDA;
        }
        g_noalloc[dev] = NoAllocEntry{id, static_cast<double*>(p)};
    }
    *out = g_noalloc[dev].ptr;
    return NACC_OK;
}
}  // namespace
}  // namespace nacc

extern "C" int nacc_update_grid_noalloc(const nacc_grid* grid, float* ema, const float* density,
                                        float decay, float thresh_frac, float thresh_abs,
                                        uint32_t* bits_out, void* stream) {
    clear_error();
    GridGeom g;
    if (!make_geom(grid, &g, false)) return NACC_ERR_INVALID_ARG;
    const int64_t n = (int64_t)g.n_levels * g.res * g.res * g.res;
    NACC_CHECK_ARG(n <= kNoAllocMaxCells,
                   "grid has %lld cells; nacc_update_grid_noalloc supports at most %lld "
                   "(use nacc_update_grid with caller scratch)",
                   (long long)n, (long long)kNoAllocMaxCells);
    NACC_CHECK_ARG(ema && density && bits_out, "ema / density / bits_out is NULL");
    NACC_CHECK_ARG(decay >= 0.0f && decay <= 1.0f, "decay=%g outside [0, 1]", (double)decay);
    NACC_CHECK_ARG(std::isfinite(thresh_frac) && std::isfinite(thresh_abs), "thresholds must be finite");
    double* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc != NACC_OK) return rc;
    // k_ema writes every partial sum it uses and k_mean_thr writes (mean,
    // threshold) before k_pack_bits reads them, so nothing needs clearing.
    double* partial = scratch;
    double* mt = scratch + kNoAllocMaxBlocks;
    return launch_update(ema, density, decay, n, (double)thresh_frac, (double)thresh_abs, bits_out, partial, mt,
                         as_stream(stream));
}

extern "C" int nacc_update_grid_frames(const nacc_grid* grid, float* ema, const float* densities, int32_t n_frames,
                                       float decay, float thresh_frac, float thresh_abs, uint32_t* bits_out,
                                       void* scratch, size_t scratch_bytes, void* stream) {
    clear_error();
    GridGeom g;
    if (!make_geom(grid, &g, false)) return NACC_ERR_INVALID_ARG;
    NACC_CHECK_ARG(ema && densities && bits_out, "ema / densities / bits_out is NULL");
    NACC_CHECK_ARG(n_frames >= 1 && n_frames <= 4096, "n_frames=%d outside [1, 4096]", n_frames);
    NACC_CHECK_ARG(decay >= 0.0f && decay <= 1.0f, "decay=%g outside [0, 1]", (double)decay);
    NACC_CHECK_ARG(std::isfinite(thresh_frac) && std::isfinite(thresh_abs), "thresholds must be finite");
    const int64_t n = (int64_t)g.n_levels * g.res * g.res * g.res;
    const size_t need = nacc_update_grid_scratch_bytes(n);
    NACC_CHECK_ARG(scratch != nullptr && scratch_bytes >= need, "scratch too small: %zu < %zu bytes", scratch_bytes,
                   need);
    NACC_CHECK_ARG((reinterpret_cast<uintptr_t>(scratch) & 255) == 0, "scratch not 256-byte aligned");
    const int64_t nb = (n + kEmaCells - 1) / kEmaCells;
    double* partial = static_cast<double*>(scratch);
    double* mt = reinterpret_cast<double*>(static_cast<char*>(scratch) + align256(sizeof(double) * (size_t)nb));
    return launch_update(ema, densities, decay, n, (double)thresh_frac, (double)thresh_abs, bits_out, partial, mt,
                         as_stream(stream), n_frames);
}

namespace nacc {
namespace {
int grid_samples_args(const nacc_grid* grid, GridGeom* g, const float* rays_o, const float* rays_d,
                      const int32_t* ray_indices, const float* t_starts, const float* t_ends,
                      const int64_t* n_samples) {
    if (!make_geom(grid, g, false)) return NACC_ERR_INVALID_ARG;
    NACC_CHECK_ARG(rays_o && rays_d && ray_indices && t_starts && t_ends && n_samples, "a pointer argument is NULL");
    return NACC_OK;
}
}  // namespace
}  // namespace nacc

extern "C" int nacc_grid_density_lookup(const nacc_grid* grid, const float* density, const float* rays_o,
                                        const float* rays_d, const int32_t* ray_indices, const float* t_starts,
                                        const float* t_ends, const int64_t* n_samples, float* sigma_out,
                                        void* stream) {
    clear_error();
    GridGeom g;
    int rc = grid_samples_args(grid, &g, rays_o, rays_d, ray_indices, t_starts, t_ends, n_samples);
    if (rc != NACC_OK) return rc;
    NACC_CHECK_ARG(density && sigma_out, "density / sigma_out is NULL");
    k_grid_samples<false><<<sm_count() * 8, 256, 0, as_stream(stream)>>>(g, rays_o, rays_d, ray_indices, t_starts,
                                                                        t_ends, n_samples, density, sigma_out);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}

extern "C" int nacc_grid_density_backward(const nacc_grid* grid, const float* rays_o, const float* rays_d,
                                          const int32_t* ray_indices, const float* t_starts, const float* t_ends,
                                          const int64_t* n_samples, const float* g_sigma, float* g_density,
                                          void* stream) {
    clear_error();
    GridGeom g;
    int rc = grid_samples_args(grid, &g, rays_o, rays_d, ray_indices, t_starts, t_ends, n_samples);
    if (rc != NACC_OK) return rc;
    NACC_CHECK_ARG(g_sigma && g_density, "g_sigma / g_density is NULL");
    k_grid_samples<true><<<sm_count() * 8, 256, 0, as_stream(stream)>>>(g, rays_o, rays_d, ray_indices, t_starts,
                                                                       t_ends, n_samples, g_sigma, g_density);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}

extern "C" int nacc_update_grid_sgd(const nacc_grid* grid, float* density, float* g_density, float lr, float thresh,
                                    uint32_t* bits_out, void* stream) {
    clear_error();
    GridGeom g;
    if (!make_geom(grid, &g, false)) return NACC_ERR_INVALID_ARG;
    NACC_CHECK_ARG(density && g_density && bits_out, "density / g_density / bits_out is NULL");
    NACC_CHECK_ARG(std::isfinite(lr) && std::isfinite(thresh), "lr / thresh must be finite");
    const int64_t n = (int64_t)g.n_levels * g.res * g.res * g.res;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 16);
    k_grid_sgd<<<blocks, 256, 0, as_stream(stream)>>>(density, g_density, n, lr, thresh, bits_out);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}
