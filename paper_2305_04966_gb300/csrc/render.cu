// render.cu -- differentiable volume rendering of packed samples
// (nacc_render_fwd, nacc_render_bwd).
//
// Eq. 2 discretised (T_i = exp(-sum_{j<i} sigma_j dt_j), w_i = T_i(1 -
// exp(-sigma_i dt_i))), Table 1 "PDF Approaches" row, Algorithm 1
// "rendering", Sec. 4.2 "No Gradient Filtering" (mask T < eps).
//
// Work decomposition (no inter-CTA communication, no spin-waits):
//   * sample space is cut into fixed chunks of kChunk samples; a ray belongs
//     to the chunk holding its first sample (its CSR offset), so every ray is
//     owned by exactly one chunk; CTAs stride over chunks (persistent grid of
//     SMs x resident CTAs);
//   * within a chunk, owned rays are packed greedily into tiles of whole
//     rays of at most kTile samples; a tile is staged in shared memory with
//     coalesced loads (padded planes, conflict-free blocked reads) and every
//     thread then owns kItems consecutive samples;
//   * per-ray prefix quantities are block-wide segmented scans (head flags
//     from the CSR offsets): a forward scan of optical depth gives T_i and
//     the mask; a forward segmented sum gives the colour/opacity/depth
//     totals; for the adjoint a reverse segmented scan gives the suffix sums
//     S^c_i, S^m_i directly (no cancellation, no saved per-sample T);
//   * a ray longer than kTile is processed alone by the CTA in kTile pieces
//     carrying the scan state between pieces (the adjoint then uses
//     suffix = total - inclusive prefix, two passes over the ray).
// The tiling depends only on the offsets, so forward and adjoint see the
// same tiles and bit-identical transmittance and masks.
#include "nacc_internal.cuh"

namespace nacc {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;   // samples per staged tile
constexpr int kWarps = kThreads / 32;
constexpr int kPlane = kTile + kTile / 32;  // padded plane (one pad word per 32)
constexpr int kWin = kThreads - 1;          // rays per offsets window
constexpr int64_t kChunk = 8192;            // ray-ownership chunk (samples)

__device__ __forceinline__ int pad(int i) { return i + (i >> 5); }

struct Smem {
    float t0[kPlane];
    float t1[kPlane];
    float sg[kPlane];
    float c[3 * (kPlane + 1)];  // r, g, b planes (stride kPlane+1: distinct banks)
    int seg[kPlane];            // local ray id at the first sample of a ray, else -1
    long long off[kWin + 1];
    float wred[kWarps * 8];
    int wredi[kWarps];
    long long bcast;
};

struct RArgs {
    int64_t n_rays;
    const int64_t* off;
    const float* t0;
    const float* t1;
    const float* sg;
    const float* rgb;
    float bg0, bg1, bg2;
    float thr;  // optical-depth mask threshold (+inf: no mask)
    // forward outputs
    float* rgb_out;
    float* op_out;
    float* dep_out;
    float* tr_out;
    float* w_out;
    // adjoint
    const float* g_rgb;
    const float* g_op;
    const float* g_dep;
    float* g_sg;
    float* g_c;
};

// ---------------------------------------------------------------------------
// segmented scan states
// ---------------------------------------------------------------------------

// optical depth with a copied ray id; flag <=> rid >= 0
struct SR {
    float v;
    int rid;
};
__device__ __forceinline__ SR comb(const SR& a, const SR& b) {
    if (b.rid >= 0) return b;
    return SR{a.v + b.v, a.rid};
}
__device__ __forceinline__ SR shfl_up(const SR& x, int o) {
    return SR{__shfl_up_sync(0xffffffffu, x.v, o), __shfl_up_sync(0xffffffffu, x.rid, o)};
}
__device__ __forceinline__ SR shfl_down(const SR& x, int o) {
    return SR{__shfl_down_sync(0xffffffffu, x.v, o), __shfl_down_sync(0xffffffffu, x.rid, o)};
}

// K segmented sums with a flag
template <int K>
struct SS {
    float v[K];
    int f;
};
template <int K>
__device__ __forceinline__ SS<K> comb(const SS<K>& a, const SS<K>& b) {
    if (b.f) return b;
    SS<K> r;
#pragma unroll
    for (int k = 0; k < K; ++k) r.v[k] = a.v[k] + b.v[k];
    r.f = a.f;
    return r;
}
template <int K>
__device__ __forceinline__ SS<K> shfl_up(const SS<K>& x, int o) {
    SS<K> r;
#pragma unroll
    for (int k = 0; k < K; ++k) r.v[k] = __shfl_up_sync(0xffffffffu, x.v[k], o);
    r.f = __shfl_up_sync(0xffffffffu, x.f, o);
    return r;
}
template <int K>
__device__ __forceinline__ SS<K> shfl_down(const SS<K>& x, int o) {
    SS<K> r;
#pragma unroll
    for (int k = 0; k < K; ++k) r.v[k] = __shfl_down_sync(0xffffffffu, x.v[k], o);
    r.f = __shfl_down_sync(0xffffffffu, x.f, o);
    return r;
}
template <int K>
__device__ __forceinline__ SS<K> ss_zero(int f) {
    SS<K> r;
#pragma unroll
    for (int k = 0; k < K; ++k) r.v[k] = 0.0f;
    r.f = f;
    return r;
}

__device__ __forceinline__ void put(Smem& s, int w, const SR& x) {
    s.wred[w * 8] = x.v;
    s.wredi[w] = x.rid;
}
__device__ __forceinline__ SR get(const Smem& s, int w, const SR*) { return SR{s.wred[w * 8], s.wredi[w]}; }
template <int K>
__device__ __forceinline__ void put(Smem& s, int w, const SS<K>& x) {
#pragma unroll
    for (int k = 0; k < K; ++k) s.wred[w * 8 + k] = x.v[k];
    s.wredi[w] = x.f;
}
template <int K>
__device__ __forceinline__ SS<K> get(const Smem& s, int w, const SS<K>*) {
    SS<K> r;
#pragma unroll
    for (int k = 0; k < K; ++k) r.v[k] = s.wred[w * 8 + k];
    r.f = s.wredi[w];
    return r;
}

// Block-wide exclusive scan of per-thread aggregates (thread order = sample
// order).  Returns the combination of all earlier threads' aggregates.
template <class T>
__device__ __forceinline__ T block_excl_scan(Smem& s, T x, const T& ident) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = shfl_up(inc, o);
        if (lane >= o) inc = comb(y, inc);
    }
    T exw = shfl_up(inc, 1);
    if (lane == 0) exw = ident;
    if (lane == 31) put(s, wid, inc);
    __syncthreads();
    T wp = ident;
    for (int w = 0; w < wid; ++w) wp = comb(wp, get(s, w, (const T*)nullptr));
    __syncthreads();
    return comb(wp, exw);
}

// Block-wide reverse exclusive scan: the combination of all later threads'
// aggregates, nearest last (combine(far, near)).
template <class T>
__device__ __forceinline__ T block_excl_rscan(Smem& s, T x, const T& ident) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = shfl_down(inc, o);
        if (lane + o < 32) inc = comb(y, inc);
    }
    T exw = shfl_down(inc, 1);
    if (lane == 31) exw = ident;
    if (lane == 0) put(s, wid, inc);
    __syncthreads();
    T wp = ident;
    for (int w = kWarps - 1; w > wid; --w) wp = comb(wp, get(s, w, (const T*)nullptr));
    __syncthreads();
    return comb(wp, exw);
}

// ---------------------------------------------------------------------------
// staging
// ---------------------------------------------------------------------------

__device__ __forceinline__ void load_tile(const RArgs& A, Smem& s, int64_t base, int n) {
    const int tid = threadIdx.x;
    float a[kItems], b[kItems], g[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        int i = tid + j * kThreads;
        if (i < n) {
            a[j] = __ldcs(A.t0 + base + i);
            b[j] = __ldcs(A.t1 + base + i);
            g[j] = __ldcs(A.sg + base + i);
        }
    }
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        int i = tid + j * kThreads;
        if (i < n) {
            s.t0[pad(i)] = a[j];
            s.t1[pad(i)] = b[j];
            s.sg[pad(i)] = g[j];
        }
    }
    const float* cp = A.rgb + 3 * base;
    const int n3 = 3 * n;
    float cv[3 * kItems];
#pragma unroll
    for (int j = 0; j < 3 * kItems; ++j) {
        int q = tid + j * kThreads;
        if (q < n3) cv[j] = __ldcs(cp + q);
    }
#pragma unroll
    for (int j = 0; j < 3 * kItems; ++j) {
        int q = tid + j * kThreads;
        if (q < n3) {
            int i = q / 3;
            int ch = q - 3 * i;
            s.c[ch * (kPlane + 1) + pad(i)] = cv[j];
        }
    }
}

__device__ __forceinline__ bool is_tail(const Smem& s, int i, int n, bool last_is_tail) {
    if (i + 1 < n) return s.seg[pad(i + 1)] >= 0;
    return last_is_tail;
}

// First ray r in [0, n_rays] with off[r] >= target (off[n_rays] >= target is
// required).  Executed by one full warp.
__device__ int64_t lower_bound_warp(const int64_t* off, int64_t n_rays, int64_t target) {
    const int lane = threadIdx.x & 31;
    int64_t lo = 0, hi = n_rays;
    while (hi - lo > 31) {
        int64_t span = hi - lo;
        int64_t p = lo + (span * (lane + 1)) / 32;
        bool ge = __ldg(&off[p]) >= target;
        unsigned m = __ballot_sync(0xffffffffu, ge);
        int f = __ffs(m) - 1;
        int64_t nhi = lo + (span * (f + 1)) / 32;
        int64_t nlo = f > 0 ? lo + (span * f) / 32 + 1 : lo;
        lo = nlo;
        hi = nhi;
    }
    int64_t p = lo + lane;
    bool ge = (p <= hi) && __ldg(&off[p]) >= target;
    unsigned m = __ballot_sync(0xffffffffu, ge);
    return lo + (__ffs(m) - 1);
}

// ---------------------------------------------------------------------------
// forward tile: modes
// ---------------------------------------------------------------------------
enum { kFwd = 0, kTotals = 1, kLongGrad = 2 };

struct Carry {
    float P;      // optical depth of the open segment (all samples)
    float acc[6]; // sum w c_r, w c_g, w c_b, w, w m, tau over unmasked samples
};

// Processes a staged tile of n samples starting at global sample `base`.
// Local ray ids in s.seg are relative to ray r0.  `head0` false: item 0
// continues a segment whose state is `carry` (long rays).  `last_tail`:
// the last item ends its ray.  Returns (in `carry`) the state after the
// last item.  kLongGrad uses `tot` (colour/depth/depth-sum totals of the
// ray) to form suffix sums.
template <int MODE>
__device__ void fwd_tile(const RArgs& A, Smem& s, int64_t base, int n, int64_t r0, Carry& carry,
                         bool last_tail, const float* tot) {
    const int tid = threadIdx.x;
    const int i0 = tid * kItems;
    // pass 1: optical depth scan
    float tau[kItems], P[kItems];
    int rid[kItems];
    SR agg{0.0f, -1};
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        int i = i0 + j;
        tau[j] = 0.0f;
        if (i < n) {
            float dt = __fsub_rn(s.t1[pad(i)], s.t0[pad(i)]);
            tau[j] = __fmul_rn(s.sg[pad(i)], dt);
            int sv = s.seg[pad(i)];
            if (sv >= 0) agg = SR{0.0f, sv};
            agg.v = agg.v + tau[j];
        }
    }
    SR cin{carry.P, 0};
    SR ex = comb(cin, block_excl_scan(s, agg, SR{0.0f, -1}));
    float incl_end;  // optical depth after this thread's last item
    {
        float run = ex.v;
        int cur = ex.rid;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            int i = i0 + j;
            if (i < n) {
                int sv = s.seg[pad(i)];
                if (sv >= 0) {
                    run = 0.0f;
                    cur = sv;
                }
            }
            P[j] = run;
            rid[j] = cur;
            run = run + tau[j];
        }
        incl_end = run;
    }
    // pass 2: weights and per-thread segmented sums
    float w[kItems];
    SS<6> a6 = ss_zero<6>(0);
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        int i = i0 + j;
        w[j] = 0.0f;
        if (i < n) {
            bool kept = !(P[j] > A.thr);
            if (kept) w[j] = expf(-P[j]) * -expm1f(-tau[j]);
            if (s.seg[pad(i)] >= 0) a6 = ss_zero<6>(1);
            float m = 0.5f * (s.t0[pad(i)] + s.t1[pad(i)]);
            a6.v[0] += w[j] * s.c[pad(i)];
            a6.v[1] += w[j] * s.c[(kPlane + 1) + pad(i)];
            a6.v[2] += w[j] * s.c[2 * (kPlane + 1) + pad(i)];
            a6.v[3] += w[j];
            a6.v[4] += w[j] * m;
            a6.v[5] += kept ? tau[j] : 0.0f;
        }
    }
    SS<6> cin6;
#pragma unroll
    for (int k = 0; k < 6; ++k) cin6.v[k] = carry.acc[k];
    cin6.f = 1;
    SS<6> ex6 = comb(cin6, block_excl_scan(s, a6, ss_zero<6>(0)));
    // pass 3: running inclusive sums; outputs at ray ends
    SS<6> run = ex6;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        int i = i0 + j;
        if (i < n) {
            if (s.seg[pad(i)] >= 0) run = ss_zero<6>(1);
            float cr = s.c[pad(i)], cg = s.c[(kPlane + 1) + pad(i)], cb = s.c[2 * (kPlane + 1) + pad(i)];
            float m = 0.5f * (s.t0[pad(i)] + s.t1[pad(i)]);
            bool kept = !(P[j] > A.thr);
            run.v[0] += w[j] * cr;
            run.v[1] += w[j] * cg;
            run.v[2] += w[j] * cb;
            run.v[3] += w[j];
            run.v[4] += w[j] * m;
            run.v[5] += kept ? tau[j] : 0.0f;
            if (MODE == kFwd) {
                if (A.w_out) s.sg[pad(i)] = w[j];
                if (is_tail(s, i, n, last_tail)) {
                    int64_t ray = r0 + rid[j];
                    float TN = expf(-run.v[5]);
                    A.rgb_out[3 * ray + 0] = run.v[0] + TN * A.bg0;
                    A.rgb_out[3 * ray + 1] = run.v[1] + TN * A.bg1;
                    A.rgb_out[3 * ray + 2] = run.v[2] + TN * A.bg2;
                    A.op_out[ray] = run.v[3];
                    A.dep_out[ray] = run.v[4];
                    A.tr_out[ray] = TN;
                }
            } else if (MODE == kLongGrad) {
                // suffix sums from the ray totals (long rays only)
                int64_t ray = r0;
                float gC0 = A.g_rgb ? __ldg(&A.g_rgb[3 * ray + 0]) : 0.0f;
                float gC1 = A.g_rgb ? __ldg(&A.g_rgb[3 * ray + 1]) : 0.0f;
                float gC2 = A.g_rgb ? __ldg(&A.g_rgb[3 * ray + 2]) : 0.0f;
                float gA = A.g_op ? __ldg(&A.g_op[ray]) : 0.0f;
                float gD = A.g_dep ? __ldg(&A.g_dep[ray]) : 0.0f;
                float gs = 0.0f, g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
                if (kept) {
                    float TN = expf(-tot[5]);
                    float Tn = expf(-(P[j] + tau[j]));
                    float S0 = tot[0] - run.v[0], S1 = tot[1] - run.v[1], S2 = tot[2] - run.v[2];
                    float Sm = tot[4] - run.v[4];
                    float dt = __fsub_rn(s.t1[pad(i)], s.t0[pad(i)]);
                    float g = gC0 * (Tn * cr - S0 - TN * A.bg0) + gC1 * (Tn * cg - S1 - TN * A.bg1) +
                              gC2 * (Tn * cb - S2 - TN * A.bg2) + gA * TN + gD * (Tn * m - Sm);
                    gs = dt * g;
                    g0 = w[j] * gC0;
                    g1 = w[j] * gC1;
                    g2 = w[j] * gC2;
                }
                s.sg[pad(i)] = gs;
                s.c[pad(i)] = g0;
                s.c[(kPlane + 1) + pad(i)] = g1;
                s.c[2 * (kPlane + 1) + pad(i)] = g2;
            }
        }
    }
    // state after the last item (for long rays)
    __syncthreads();
    const int owner = (n - 1) / kItems;
    if (tid == owner) {
        s.wred[0] = incl_end;
#pragma unroll
        for (int k = 0; k < 6; ++k) s.wred[1 + k] = run.v[k];
    }
    __syncthreads();
    carry.P = s.wred[0];
#pragma unroll
    for (int k = 0; k < 6; ++k) carry.acc[k] = s.wred[1 + k];
    __syncthreads();
}

// adjoint of a tile of whole rays (reverse segmented scan for the suffixes)
__device__ void bwd_tile(const RArgs& A, Smem& s, int n, int64_t r0) {
    const int tid = threadIdx.x;
    const int i0 = tid * kItems;
    float tau[kItems], P[kItems];
    int rid[kItems];
    SR agg{0.0f, -1};
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        int i = i0 + j;
        tau[j] = 0.0f;
        if (i < n) {
            float dt = __fsub_rn(s.t1[pad(i)], s.t0[pad(i)]);
            tau[j] = __fmul_rn(s.sg[pad(i)], dt);
            int sv = s.seg[pad(i)];
            if (sv >= 0) agg = SR{0.0f, sv};
            agg.v = agg.v + tau[j];
        }
    }
    SR ex = comb(SR{0.0f, 0}, block_excl_scan(s, agg, SR{0.0f, -1}));
    {
        float run = ex.v;
        int cur = ex.rid;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            int i = i0 + j;
            if (i < n) {
                int sv = s.seg[pad(i)];
                if (sv >= 0) {
                    run = 0.0f;
                    cur = sv;
                }
            }
            P[j] = run;
            rid[j] = cur;
            run = run + tau[j];
        }
    }
    // weights and the per-thread reverse aggregate of (w c, w m, kept tau)
    float w[kItems];
    SS<5> a5 = ss_zero<5>(0);
#pragma unroll
    for (int j = kItems - 1; j >= 0; --j) {
        int i = i0 + j;
        w[j] = 0.0f;
        if (i < n) {
            bool kept = !(P[j] > A.thr);
            if (kept) w[j] = expf(-P[j]) * -expm1f(-tau[j]);
            if (is_tail(s, i, n, true)) a5 = ss_zero<5>(1);
            float m = 0.5f * (s.t0[pad(i)] + s.t1[pad(i)]);
            a5.v[0] += w[j] * s.c[pad(i)];
            a5.v[1] += w[j] * s.c[(kPlane + 1) + pad(i)];
            a5.v[2] += w[j] * s.c[2 * (kPlane + 1) + pad(i)];
            a5.v[3] += w[j] * m;
            a5.v[4] += kept ? tau[j] : 0.0f;
        }
    }
    SS<5> ex5 = block_excl_rscan(s, a5, ss_zero<5>(0));
    SS<5> run = ex5;
#pragma unroll
    for (int j = kItems - 1; j >= 0; --j) {
        int i = i0 + j;
        if (i < n) {
            if (is_tail(s, i, n, true)) run = ss_zero<5>(1);
            float cr = s.c[pad(i)], cg = s.c[(kPlane + 1) + pad(i)], cb = s.c[2 * (kPlane + 1) + pad(i)];
            float m = 0.5f * (s.t0[pad(i)] + s.t1[pad(i)]);
            bool kept = !(P[j] > A.thr);
            float gs = 0.0f, g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
            if (kept) {
                int64_t ray = r0 + rid[j];
                float gC0 = A.g_rgb ? __ldg(&A.g_rgb[3 * ray + 0]) : 0.0f;
                float gC1 = A.g_rgb ? __ldg(&A.g_rgb[3 * ray + 1]) : 0.0f;
                float gC2 = A.g_rgb ? __ldg(&A.g_rgb[3 * ray + 2]) : 0.0f;
                float gA = A.g_op ? __ldg(&A.g_op[ray]) : 0.0f;
                float gD = A.g_dep ? __ldg(&A.g_dep[ray]) : 0.0f;
                float incl = P[j] + tau[j];
                float Tn = expf(-incl);
                float TN = expf(-(incl + run.v[4]));
                float dt = __fsub_rn(s.t1[pad(i)], s.t0[pad(i)]);
                float g = gC0 * (Tn * cr - run.v[0] - TN * A.bg0) +
                          gC1 * (Tn * cg - run.v[1] - TN * A.bg1) +
                          gC2 * (Tn * cb - run.v[2] - TN * A.bg2) + gA * TN +
                          gD * (Tn * m - run.v[3]);
                gs = dt * g;
                g0 = w[j] * gC0;
                g1 = w[j] * gC1;
                g2 = w[j] * gC2;
            }
            run.v[0] += w[j] * cr;
            run.v[1] += w[j] * cg;
            run.v[2] += w[j] * cb;
            run.v[3] += w[j] * m;
            run.v[4] += kept ? tau[j] : 0.0f;
            // each thread only ever reads its own items of these planes
            s.sg[pad(i)] = gs;
            s.c[pad(i)] = g0;
            s.c[(kPlane + 1) + pad(i)] = g1;
            s.c[2 * (kPlane + 1) + pad(i)] = g2;
        }
    }
}

// coalesced write-back of the per-sample adjoint (planes sg, c)
__device__ __forceinline__ void store_grads(const RArgs& A, Smem& s, int64_t base, int n) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        int i = tid + j * kThreads;
        if (i < n) __stcs(A.g_sg + base + i, s.sg[pad(i)]);
    }
    float* cp = A.g_c + 3 * base;
    const int n3 = 3 * n;
#pragma unroll
    for (int j = 0; j < 3 * kItems; ++j) {
        int q = tid + j * kThreads;
        if (q < n3) {
            int i = q / 3;
            int ch = q - 3 * i;
            __stcs(cp + q, s.c[ch * (kPlane + 1) + pad(i)]);
        }
    }
}

__device__ __forceinline__ void store_weights(const RArgs& A, Smem& s, int64_t base, int n) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        int i = tid + j * kThreads;
        if (i < n) __stcs(A.w_out + base + i, s.sg[pad(i)]);
    }
}

// clear seg for n items, mark a single head at item 0 if head0
__device__ __forceinline__ void set_single_segment(Smem& s, int n, bool head0) {
    for (int i = threadIdx.x; i < n; i += kThreads) s.seg[pad(i)] = -1;
    __syncthreads();
    if (threadIdx.x == 0 && head0) s.seg[0] = 0;
}

// A ray longer than one tile: pieces of kTile with carried state.
template <bool kBwd>
__device__ void long_ray(const RArgs& A, Smem& s, int64_t ray, int64_t b, int64_t e) {
    const int64_t len = e - b;
    Carry cr;
    cr.P = 0.0f;
#pragma unroll
    for (int k = 0; k < 6; ++k) cr.acc[k] = 0.0f;
    if (!kBwd) {
        for (int64_t p = 0; p < len; p += kTile) {
            int n = (int)min64(kTile, len - p);
            set_single_segment(s, n, p == 0);
            load_tile(A, s, b + p, n);
            __syncthreads();
            fwd_tile<kFwd>(A, s, b + p, n, ray, cr, p + n == len, nullptr);
            if (A.w_out) store_weights(A, s, b + p, n);
            __syncthreads();
        }
    } else {
        // pass 1: totals
        for (int64_t p = 0; p < len; p += kTile) {
            int n = (int)min64(kTile, len - p);
            set_single_segment(s, n, p == 0);
            load_tile(A, s, b + p, n);
            __syncthreads();
            fwd_tile<kTotals>(A, s, b + p, n, ray, cr, p + n == len, nullptr);
        }
        float tot[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) tot[k] = cr.acc[k];
        cr.P = 0.0f;
#pragma unroll
        for (int k = 0; k < 6; ++k) cr.acc[k] = 0.0f;
        // pass 2: gradients with suffix = total - inclusive prefix
        for (int64_t p = 0; p < len; p += kTile) {
            int n = (int)min64(kTile, len - p);
            set_single_segment(s, n, p == 0);
            load_tile(A, s, b + p, n);
            __syncthreads();
            fwd_tile<kLongGrad>(A, s, b + p, n, ray, cr, p + n == len, tot);
            store_grads(A, s, b + p, n);
            __syncthreads();
        }
    }
}

template <bool kBwd>
__global__ void __launch_bounds__(kThreads, 2) k_render(RArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& s = *reinterpret_cast<Smem*>(smem_raw);
    const int tid = threadIdx.x;
    const int64_t S = __ldg(&A.off[A.n_rays]);
    const int64_t nchunks = S / kChunk + 1;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int64_t hi_s = (c + 1) * kChunk;
        if (tid < 32) {
            int64_t r = lower_bound_warp(A.off, A.n_rays, c * kChunk);
            if (tid == 0) s.bcast = r;
        }
        __syncthreads();
        int64_t r = s.bcast;
        __syncthreads();
        while (r < A.n_rays) {
            const int64_t nwin = min64(kWin, A.n_rays - r);
            if (tid <= nwin) s.off[tid] = __ldg(&A.off[r + tid]);
            __syncthreads();
            int n_owned = __syncthreads_count(tid < nwin && s.off[tid] < hi_s);
            if (n_owned == 0) break;
            int n_fit = __syncthreads_count(tid <= n_owned && s.off[tid] - s.off[0] <= kTile);
            const int e = n_fit - 1;
            if (e == 0) {
                const int64_t b = s.off[0], en = s.off[1];
                __syncthreads();
                long_ray<kBwd>(A, s, r, b, en);
                r += 1;
                continue;
            }
            const int64_t base = s.off[0];
            const int n = (int)(s.off[e] - base);
            for (int i = tid; i < n; i += kThreads) s.seg[pad(i)] = -1;
            __syncthreads();
            if (tid < e) {
                const long long a = s.off[tid], bnd = s.off[tid + 1];
                if (bnd > a) {
                    s.seg[pad((int)(a - base))] = tid;
                } else if (!kBwd) {
                    const int64_t ray = r + tid;
                    A.rgb_out[3 * ray + 0] = A.bg0;
                    A.rgb_out[3 * ray + 1] = A.bg1;
                    A.rgb_out[3 * ray + 2] = A.bg2;
                    A.op_out[ray] = 0.0f;
                    A.dep_out[ray] = 0.0f;
                    A.tr_out[ray] = 1.0f;
                }
            }
            if (n > 0) {
                load_tile(A, s, base, n);
                __syncthreads();
                if (!kBwd) {
                    Carry cr;
                    cr.P = 0.0f;
#pragma unroll
                    for (int k = 0; k < 6; ++k) cr.acc[k] = 0.0f;
                    fwd_tile<kFwd>(A, s, base, n, r, cr, true, nullptr);
                    if (A.w_out) store_weights(A, s, base, n);
                } else {
                    bwd_tile(A, s, n, r);
                    __syncthreads();
                    store_grads(A, s, base, n);
                }
            }
            r += e;
            __syncthreads();
        }
        __syncthreads();
    }
}

int render_grid_size(bool bwd, size_t smem) {
    int per_sm = 1;
    if (bwd)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render<true>, kThreads, smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render<false>, kThreads, smem);
    if (per_sm < 1) per_sm = 1;
    return per_sm * sm_count();
}

int launch_render(bool bwd, const RArgs& A, cudaStream_t st) {
    size_t smem = sizeof(Smem);
    if (bwd)
        NACC_CUDA_TRY(cudaFuncSetAttribute(k_render<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    else
        NACC_CUDA_TRY(cudaFuncSetAttribute(k_render<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int grid = render_grid_size(bwd, smem);
    if (bwd)
        k_render<true><<<grid, kThreads, smem, st>>>(A);
    else
        k_render<false><<<grid, kThreads, smem, st>>>(A);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}

int check_common(int64_t n_rays, const int64_t* offsets, const float* t_starts, const float* t_ends,
                 const float* sigmas, const float* rgbs, const float* bg) {
    NACC_CHECK_ARG(n_rays >= 0 && n_rays < (int64_t(1) << 40), "n_rays=%lld out of range", (long long)n_rays);
    NACC_CHECK_ARG(offsets != nullptr, "offsets is NULL");
    NACC_CHECK_ARG(bg != nullptr, "bg is NULL");
    NACC_CHECK_ARG(t_starts && t_ends && sigmas && rgbs, "a sample array is NULL");
    return NACC_OK;
}

}  // namespace
}  // namespace nacc

using namespace nacc;

extern "C" int nacc_render_fwd(int64_t n_rays, const int64_t* offsets, const float* t_starts,
                               const float* t_ends, const float* sigmas, const float* rgbs,
                               const float* bg, float early_stop_eps, float* rgb_out,
                               float* opacity_out, float* depth_out, float* trans_out,
                               float* weights_out, void* stream) {
    clear_error();
    int rc = check_common(n_rays, offsets, t_starts, t_ends, sigmas, rgbs, bg);
    if (rc != NACC_OK) return rc;
    NACC_CHECK_ARG(rgb_out && opacity_out && depth_out && trans_out, "an output array is NULL");
    if (n_rays == 0) return NACC_OK;
    RArgs A{};
    A.n_rays = n_rays;
    A.off = offsets;
    A.t0 = t_starts;
    A.t1 = t_ends;
    A.sg = sigmas;
    A.rgb = rgbs;
    A.bg0 = bg[0];
    A.bg1 = bg[1];
    A.bg2 = bg[2];
    A.thr = tau_threshold(early_stop_eps);
    A.rgb_out = rgb_out;
    A.op_out = opacity_out;
    A.dep_out = depth_out;
    A.tr_out = trans_out;
    A.w_out = weights_out;
    return launch_render(false, A, as_stream(stream));
}

extern "C" int nacc_render_bwd(int64_t n_rays, const int64_t* offsets, const float* t_starts,
                               const float* t_ends, const float* sigmas, const float* rgbs,
                               const float* bg, float early_stop_eps, const float* g_rgb,
                               const float* g_opacity, const float* g_depth, float* g_sigmas,
                               float* g_rgbs, void* stream) {
    clear_error();
    int rc = check_common(n_rays, offsets, t_starts, t_ends, sigmas, rgbs, bg);
    if (rc != NACC_OK) return rc;
    NACC_CHECK_ARG(g_sigmas && g_rgbs, "g_sigmas / g_rgbs is NULL");
    if (n_rays == 0) return NACC_OK;
    RArgs A{};
    A.n_rays = n_rays;
    A.off = offsets;
    A.t0 = t_starts;
    A.t1 = t_ends;
    A.sg = sigmas;
    A.rgb = rgbs;
    A.bg0 = bg[0];
    A.bg1 = bg[1];
    A.bg2 = bg[2];
    A.thr = tau_threshold(early_stop_eps);
    A.g_rgb = g_rgb;
    A.g_op = g_opacity;
    A.g_dep = g_depth;
    A.g_sg = g_sigmas;
    A.g_c = g_rgbs;
    return launch_render(true, A, as_stream(stream));
}
