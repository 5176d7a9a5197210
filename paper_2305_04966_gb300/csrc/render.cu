// render.cu -- differentiable volume rendering of packed samples
// (nacc_render_fwd, nacc_render_bwd).
//
// Eq. 2 discretised (T_i = exp(-sum_{j<i} sigma_j dt_j), w_i = T_i(1 -
// exp(-sigma_i dt_i))), Table 1 "PDF Approaches" row, Algorithm 1
// "rendering", Sec. 4.2 "No Gradient Filtering" (mask T < eps).
//
// Warp-specialised streaming kernel (persistent: SMs x 2 CTAs of 8 warps):
//   * ray ownership: sample space is cut into fixed chunks of kChunk samples;
//     a ray belongs to the chunk holding its first sample (CSR offset); each
//     CTA takes a contiguous range of chunks.  Inside a chunk the owned rays
//     are packed greedily into tiles of whole rays spanning at most kTile
//     positions (positions count from the tile's first sample rounded down
//     to a multiple of 4, so every bulk copy and every vector store is
//     16-byte aligned) and at most kWin rays.  The tiling depends only on the
//     offsets, so forward and adjoint see identical tiles and bit-identical
//     transmittance.
//   * one producer warp plans the next tile from the offsets, then streams
//     the tile's t0, t1, sigma and rgb planes into a kStages-deep shared-
//     memory ring with 1-D bulk asynchronous copies (cp.async.bulk + mbarrier
//     transaction counts) and writes the tile's segment map (ray heads / tails
//     per position) and, for the adjoint, the rays' upstream gradients;
//   * seven consumer warps own 8 consecutive positions per thread (128-bit
//     shared loads).  The forward exclusive optical depth P_i is one
//     block-wide segmented scan.  Forward: rays that end inside a thread are
//     finished there; each thread parks the partial sums of its first and
//     last (open) segments in its own slots of the spent stage planes, and one
//     warp per ray that spans threads adds them up in a fixed order.
//     Adjoint: a reverse block-wide segmented scan gives the suffix sums
//     S^c_i, S^m_i directly (no cancellation, no saved per-sample
//     transmittance).  Per-sample results leave as aligned 128-bit global
//     stores straight from registers;
//   * a ray longer than one tile is streamed alone in pieces with the scan
//     state carried between pieces (the adjoint then takes two passes and
//     forms suffixes as total - inclusive prefix on those rays only).
// Every wait is bounded (2 s of %globaltimer); on expiry the kernel records
// NACC_ERR_TIMEOUT in a device status word (nacc_device_status) and returns
// after its own copies have landed.
#include "async_copy.cuh"
#include "nacc_internal.cuh"

// bit 0: a bounded wait expired in a render kernel
__device__ unsigned int g_nacc_render_status;

namespace nacc {
namespace {

constexpr int kConsumerWarps = 7;  // + 1 producer = 8 warps: 2 CTAs/SM at 128 registers
constexpr int kConsumers = kConsumerWarps * 32;
constexpr int kThreads = kConsumers + 32;   // + one producer warp
constexpr int kItems = 8;                   // consecutive positions per consumer thread
constexpr int kTile = kConsumers * kItems;  // positions per stage
constexpr int kStages = 2;
constexpr int kWin = 127;                   // rays per tile at most
constexpr int64_t kChunk = 8192;            // ray-ownership chunk (samples)
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr int kBarConsumers = 1;

enum : int { kKindTile = 0, kKindLong = 1, kKindDone = 2 };
enum : int { kFirst = 1, kLast = 2, kPass2 = 4 };

struct StageDesc {
    long long base;   // first sample of the tile / piece
    long long abase;  // base rounded down to a multiple of 4 = position 0
    long long cend;   // end (exclusive) of the bulk-copied range
    long long r0;     // first ray of the tile / the long ray
    int n;            // samples
    int e;            // rays in the tile
    int kind;
    int flags;
    short off_rel[kWin + 1];  // tile: offsets[r0 + j] - abase, j = 0..e
};

struct alignas(128) Stage {
    float t0[kTile];
    float t1[kTile];
    float sg[kTile];
    float c[3 * kTile];
    unsigned short seg[kTile];  // low byte: head local id + 1, high byte: tail local id + 1
    StageDesc d;
};

template <bool kBwd>
struct Smem {
    Stage st[kStages];
    float pray[kBwd ? kStages : 1][kBwd ? kWin * 5 : 1];  // adjoint: per-ray g_rgb (3), g_A, g_D
    uint64_t full[kStages];
    uint64_t empty[kStages];
    float wred[2][kConsumerWarps * 8];  // warp aggregates, double-buffered
    int wredi[2][kConsumerWarps];
    float carry[8];
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
    float* rgb_out;
    float* op_out;
    float* dep_out;
    float* tr_out;
    float* w_out;
    const float* g_rgb;
    const float* g_op;
    const float* g_dep;
    float* g_sg;
    float* g_c;
};

__device__ __forceinline__ void report_timeout() { atomicOr(&g_nacc_render_status, 1u); }

__device__ __forceinline__ void consumer_sync() { named_barrier(kBarConsumers, kConsumers); }

// AND of `pred` over the consumer threads (also a barrier for them).
__device__ __forceinline__ bool consumer_all(bool pred) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.s32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\t"
        "selp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((int)pred), "r"(kBarConsumers), "r"(kConsumers)
        : "memory");
    return r != 0;
}

// ---------------------------------------------------------------------------
// segmented scan state: K sums and a segment id; "starts a segment" <=> id >= 0
// ---------------------------------------------------------------------------
template <int K>
struct Seg {
    float v[K];
    int id;
};
template <int K>
__device__ __forceinline__ Seg<K> seg_zero(int id) {
    Seg<K> r;
#pragma unroll
    for (int k = 0; k < K; ++k) r.v[k] = 0.0f;
    r.id = id;
    return r;
}
// a precedes b in scan order: b wins if it starts a segment, else sums.
template <int K>
__device__ __forceinline__ Seg<K> comb(const Seg<K>& a, const Seg<K>& b) {
    if (b.id >= 0) return b;
    Seg<K> r;
#pragma unroll
    for (int k = 0; k < K; ++k) r.v[k] = a.v[k] + b.v[k];
    r.id = a.id;
    return r;
}
template <int K, bool kUp>
__device__ __forceinline__ Seg<K> shfl(const Seg<K>& x, int o) {
    Seg<K> r;
#pragma unroll
    for (int k = 0; k < K; ++k)
        r.v[k] = kUp ? __shfl_up_sync(0xffffffffu, x.v[k], o) : __shfl_down_sync(0xffffffffu, x.v[k], o);
    r.id = kUp ? __shfl_up_sync(0xffffffffu, x.id, o) : __shfl_down_sync(0xffffffffu, x.id, o);
    return r;
}

// Exclusive segmented scan over the consumer threads, forward (thread order)
// or reverse; one barrier; `buf` alternates between consecutive scans.
template <int K, bool kForward, class SM>
__device__ __forceinline__ Seg<K> block_scan(SM& s, const Seg<K>& x, int buf) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    Seg<K> inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        Seg<K> y = shfl<K, kForward>(inc, o);
        if (kForward ? lane >= o : lane + o < 32) inc = comb(y, inc);
    }
    Seg<K> exw = shfl<K, kForward>(inc, 1);
    if (kForward ? lane == 0 : lane == 31) exw = seg_zero<K>(-1);
    if (kForward ? lane == 31 : lane == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) s.wred[buf][wid * 8 + k] = inc.v[k];
        s.wredi[buf][wid] = inc.id;
    }
    consumer_sync();
    Seg<K> wp = seg_zero<K>(-1);
#pragma unroll
    for (int q = 0; q < kConsumerWarps; ++q) {
        const int w = kForward ? q : kConsumerWarps - 1 - q;
        Seg<K> g;
#pragma unroll
        for (int k = 0; k < K; ++k) g.v[k] = s.wred[buf][w * 8 + k];
        g.id = s.wredi[buf][w];
        if (kForward ? w < wid : w > wid) wp = comb(wp, g);
    }
    return comb(wp, exw);
}

// 1 - exp(-x) for x >= 0: Taylor series x(1 - x/2(1 - x/3(1 - x/4(1 - x/5))))
// below 1/16 (truncation < 2e-9 relative), else 1 - exp(-x) directly.
__device__ __forceinline__ float one_minus_exp_neg(float x) {
    const float ser = x * (1.0f - 0.5f * x * (1.0f - x * (1.0f / 3.0f) * (1.0f - 0.25f * x * (1.0f - 0.2f * x))));
    const float dir = 1.0f - __expf(-x);
    return x < 0.0625f ? ser : dir;
}

__device__ __forceinline__ void ld8(const float* plane, int p, float v[8]) {
    const float4 a = *reinterpret_cast<const float4*>(plane + p);
    const float4 b = *reinterpret_cast<const float4*>(plane + p + 4);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
    v[4] = b.x;
    v[5] = b.y;
    v[6] = b.z;
    v[7] = b.w;
}

// colours of 8 consecutive positions: 24 floats, 6 x 128-bit
__device__ __forceinline__ void ld24(const float* c, int p, float v[24]) {
    const float4* q = reinterpret_cast<const float4*>(c + 3 * p);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float4 a = q[k];
        v[4 * k + 0] = a.x;
        v[4 * k + 1] = a.y;
        v[4 * k + 2] = a.z;
        v[4 * k + 3] = a.w;
    }
}

// Per-thread view of the segment map of its 8 positions.
struct SegView {
    uint4 raw;
    unsigned head;   // bit j: position j starts a ray
    unsigned tail;   // bit j: position j ends a ray
    unsigned valid;  // bit j: position j belongs to the tile
};
__device__ __forceinline__ unsigned seg_entry(const uint4& s, int j) {
    const unsigned w = j < 2 ? s.x : j < 4 ? s.y : j < 6 ? s.z : s.w;
    return (j & 1) ? (w >> 16) : (w & 0xffffu);
}
__device__ __forceinline__ SegView seg_view(const unsigned short* seg, int p0, int o_rel, int pend) {
    SegView v;
    v.raw = *reinterpret_cast<const uint4*>(seg + p0);
    v.head = 0;
    v.tail = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const unsigned e = seg_entry(v.raw, j);
        v.head |= ((e & 0xffu) != 0u) << j;
        v.tail |= ((e >> 8) != 0u) << j;
    }
    const int lo = min(max(o_rel - p0, 0), 8), hi = min(max(pend - p0, 0), 8);
    v.valid = ((1u << hi) - 1u) & ~((1u << lo) - 1u);
    return v;
}
__device__ __forceinline__ int tail_id(const SegView& v, int j) { return (int)(seg_entry(v.raw, j) >> 8) - 1; }

// Store 8 consecutive results of positions [p, p+8) to dst[abase + p ..]
// (vector stores when all 8 are valid, else per element).
__device__ __forceinline__ void st8_global(float* dst, long long abase, int p, unsigned valid, const float v[8]) {
    float* d = dst + abase + p;
    if (valid == 0xffu) {
        __stcs(reinterpret_cast<float4*>(d), make_float4(v[0], v[1], v[2], v[3]));
        __stcs(reinterpret_cast<float4*>(d) + 1, make_float4(v[4], v[5], v[6], v[7]));
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (valid & (1u << j)) __stcs(d + j, v[j]);
    }
}
__device__ __forceinline__ void st24_global(float* dst, long long abase, int p, unsigned valid, const float v[24]) {
    float* d = dst + 3 * (abase + p);
    if (valid == 0xffu) {
#pragma unroll
        for (int k = 0; k < 6; ++k)
            __stcs(reinterpret_cast<float4*>(d) + k, make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]));
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (valid & (1u << j)) {
                __stcs(d + 3 * j + 0, v[3 * j + 0]);
                __stcs(d + 3 * j + 1, v[3 * j + 1]);
                __stcs(d + 3 * j + 2, v[3 * j + 2]);
            }
    }
}

__device__ __forceinline__ void write_ray(const RArgs& A, long long ray, const float v[6]) {
    const float TN = __expf(-v[5]);
    A.rgb_out[3 * ray + 0] = v[0] + TN * A.bg0;
    A.rgb_out[3 * ray + 1] = v[1] + TN * A.bg1;
    A.rgb_out[3 * ray + 2] = v[2] + TN * A.bg2;
    A.op_out[ray] = v[3];
    A.dep_out[ray] = v[4];
    A.tr_out[ray] = TN;
}

// ---------------------------------------------------------------------------
// producer warp
// ---------------------------------------------------------------------------

// First ray r in [0, n_rays] with off[r] >= target (off[n_rays] >= target).
__device__ int64_t lower_bound_warp(const int64_t* off, int64_t n_rays, int64_t target) {
    const int lane = threadIdx.x & 31;
    int64_t lo = 0, hi = n_rays;
    while (hi - lo > 31) {
        const int64_t span = hi - lo;
        const int64_t p = lo + (span * (lane + 1)) / 32;
        const bool ge = __ldg(&off[p]) >= target;
        const unsigned m = __ballot_sync(0xffffffffu, ge);
        const int f = __ffs(m) - 1;
        const int64_t nhi = lo + (span * (f + 1)) / 32;
        const int64_t nlo = f > 0 ? lo + (span * f) / 32 + 1 : lo;
        lo = nlo;
        hi = nhi;
    }
    const int64_t p = lo + lane;
    const bool ge = (p <= hi) && __ldg(&off[p]) >= target;
    const unsigned m = __ballot_sync(0xffffffffu, ge);
    return lo + (__ffs(m) - 1);
}

template <bool kBwd>
struct Producer {
    const RArgs& A;
    Smem<kBwd>& s;
    long long S4;  // total samples rounded down to a multiple of 4
    int it;        // stages issued so far
    bool ok;

    // Wait (all lanes, bounded) until the stage of issue `it` is free.
    __device__ bool acquire(int& stg) {
        stg = it % kStages;
        const uint32_t ph = (uint32_t)(it / kStages) & 1u;
        bool got = true;
        if (it >= kStages) got = mbar_wait_bounded(&s.empty[stg], ph ^ 1u, kWaitLimitNs);
        return __all_sync(0xffffffffu, got);
    }

    __device__ long long copy_end(long long end) const {
        const long long ce = (end + 3) & ~3ll;
        return ce < S4 ? ce : S4;
    }

    // Lane 0: raise the stage's expected bytes and start the bulk copies of
    // positions [abase, cend) (the stage's later arrive completes the phase).
    __device__ void start_copies(int stg, long long abase, long long cend) {
        Stage& st = s.st[stg];
        if (cend > abase) {
            const uint32_t cnt = (uint32_t)(cend - abase);
            mbar_expect_tx(&s.full[stg], 24u * cnt);
            bulk_copy_g2s(st.t0, A.t0 + abase, 4u * cnt, &s.full[stg]);
            bulk_copy_g2s(st.t1, A.t1 + abase, 4u * cnt, &s.full[stg]);
            bulk_copy_g2s(st.sg, A.sg + abase, 4u * cnt, &s.full[stg]);
            bulk_copy_g2s(st.c, A.rgb + 3 * abase, 12u * cnt, &s.full[stg]);
        }
    }

    __device__ void clear_seg(Stage& st) {
        const int lane = threadIdx.x & 31;
        uint4* p = reinterpret_cast<uint4*>(st.seg);
#pragma unroll
        for (int k = 0; k < kTile / 8 / 32; ++k) p[lane + 32 * k] = make_uint4(0, 0, 0, 0);
    }

    __device__ void load_ray_grads(int stg, int j, long long ray) {
        if (kBwd) {
            float* pr = &s.pray[stg][5 * j];
            pr[0] = A.g_rgb ? __ldg(&A.g_rgb[3 * ray + 0]) : 0.0f;
            pr[1] = A.g_rgb ? __ldg(&A.g_rgb[3 * ray + 1]) : 0.0f;
            pr[2] = A.g_rgb ? __ldg(&A.g_rgb[3 * ray + 2]) : 0.0f;
            pr[3] = A.g_op ? __ldg(&A.g_op[ray]) : 0.0f;
            pr[4] = A.g_dep ? __ldg(&A.g_dep[ray]) : 0.0f;
        }
    }

    __device__ void publish(int stg) {
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(&s.full[stg]);
        __syncwarp();
        ++it;
    }

    __device__ void long_ray(int64_t ray, long long b, long long e) {
        const int lane = threadIdx.x & 31;
        for (int pass = 0; pass < (kBwd ? 2 : 1) && ok; ++pass) {
            long long p = b;
            while (p < e) {
                const long long abase = p & ~3ll;
                const long long n = min64(kTile - (p - abase), e - p);
                const long long cend = copy_end(p + n);
                int stg;
                if (!acquire(stg)) {
                    ok = false;
                    return;
                }
                Stage& st = s.st[stg];
                if (lane == 0) start_copies(stg, abase, cend);
                clear_seg(st);
                __syncwarp();
                if (lane == 0) {
                    StageDesc& d = st.d;
                    d.kind = kKindLong;
                    d.base = p;
                    d.abase = abase;
                    d.cend = cend;
                    d.r0 = ray;
                    d.n = (int)n;
                    d.e = 1;
                    d.flags = (p == b ? kFirst : 0) | (p + n == e ? kLast : 0) | (pass ? kPass2 : 0);
                    const int o = (int)(p - abase);
                    if (p == b) st.seg[o] = 1;
                    if (p + n == e) st.seg[o + n - 1] = (unsigned short)(st.seg[o + n - 1] | (1u << 8));
                    load_ray_grads(stg, 0, ray);
                }
                publish(stg);
                p += n;
            }
        }
    }

    __device__ void run(int64_t c_begin, int64_t c_end) {
        const int lane = threadIdx.x & 31;
        int64_t r = c_begin < c_end ? lower_bound_warp(A.off, A.n_rays, c_begin * kChunk) : A.n_rays;
        for (int64_t c = c_begin; c < c_end && ok; ++c) {
            const long long hi_s = (c + 1) * kChunk;
            while (r < A.n_rays && ok) {
                // plan the next tile (before waiting for a free stage)
                const int nwin = (int)min64(kWin, A.n_rays - r);
                long long v[4];  // entries j = lane*4 + q, j <= nwin
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = lane * 4 + q;
                    v[q] = j <= nwin ? __ldg(&A.off[r + j]) : 0x7fffffffffffffffll;
                }
                int own = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) own += (lane * 4 + q < nwin && v[q] < hi_s) ? 1 : 0;
                const int n_owned = __reduce_add_sync(0xffffffffu, own);
                if (n_owned == 0) break;
                const long long base = __shfl_sync(0xffffffffu, v[0], 0);
                const long long abase = base & ~3ll;
                const long long lim = abase + kTile;
                int fit = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) fit += (lane * 4 + q <= n_owned && v[q] <= lim) ? 1 : 0;
                const int e = __reduce_add_sync(0xffffffffu, fit) - 1;
                if (e == 0) {
                    const long long end = __shfl_sync(0xffffffffu, v[1], 0);
                    long_ray(r, base, end);
                    r += 1;
                    continue;
                }
                long long tend = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (lane * 4 + q == e) tend = v[q];
                tend = __shfl_sync(0xffffffffu, tend, e >> 2);
                const long long next_lane0 = __shfl_down_sync(0xffffffffu, v[0], 1);
                const long long cend = copy_end(tend);
                int stg;
                if (!acquire(stg)) {
                    ok = false;
                    break;
                }
                Stage& st = s.st[stg];
                if (lane == 0) start_copies(stg, abase, cend);
                clear_seg(st);
                __syncwarp();
                // ray j = lane*4+q (j < e): head at v[q]-abase, tail at v(j+1)-abase-1
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = lane * 4 + q;
                    if (j <= e) st.d.off_rel[j] = (short)(v[q] - abase);
                    if (j < e) {
                        const long long nx = q < 3 ? v[q + 1] : next_lane0;
                        if (nx > v[q]) {
                            const int h = (int)(v[q] - abase), t = (int)(nx - abase - 1);
                            if (h == t) {
                                st.seg[h] = (unsigned short)((j + 1) | ((j + 1) << 8));
                            } else {
                                st.seg[h] = (unsigned short)(j + 1);
                                st.seg[t] = (unsigned short)((j + 1) << 8);
                            }
                        }
                        load_ray_grads(stg, j, r + j);
                    }
                }
                if (lane == 0) {
                    StageDesc& d = st.d;
                    d.kind = kKindTile;
                    d.base = base;
                    d.abase = abase;
                    d.cend = cend;
                    d.r0 = r;
                    d.n = (int)(tend - base);
                    d.e = e;
                    d.flags = 0;
                }
                publish(stg);
                r += e;
            }
        }
        int stg;
        if (ok && acquire(stg)) {
            if (lane == 0) {
                s.st[stg].d.kind = kKindDone;
                s.st[stg].d.n = 0;
            }
            publish(stg);
        } else {
            ok = false;
        }
        if (!ok) {
            if (lane == 0) report_timeout();
            // let every copy this warp started land before the CTA can exit
            for (int k = 0; k < kStages && k < it; ++k) {
                const int i = it - 1 - k;
                mbar_wait_bounded(&s.full[i % kStages], (uint32_t)(i / kStages) & 1u, kWaitLimitNs);
            }
        }
    }
};

// ---------------------------------------------------------------------------
// consumer side
// ---------------------------------------------------------------------------

struct Carry {
    float P;       // optical depth after the last item processed (all samples)
    float acc[6];  // sum w c_r, w c_g, w c_b, w, w m, unmasked tau
};

// Loads positions of [max(cend, base), base + n) -- the ragged end of the
// arrays that the bulk copy left out -- with plain loads.
__device__ __forceinline__ void load_ragged_end(const RArgs& A, Stage& st) {
    const long long from = st.d.cend > st.d.base ? st.d.cend : st.d.base;
    const long long to = st.d.base + st.d.n;
    for (long long i = from + threadIdx.x; i < to; i += kConsumers) {
        const int p = (int)(i - st.d.abase);
        st.t0[p] = __ldg(A.t0 + i);
        st.t1[p] = __ldg(A.t1 + i);
        st.sg[p] = __ldg(A.sg + i);
        st.c[3 * p + 0] = __ldg(A.rgb + 3 * i + 0);
        st.c[3 * p + 1] = __ldg(A.rgb + 3 * i + 1);
        st.c[3 * p + 2] = __ldg(A.rgb + 3 * i + 2);
    }
}

// Pass 1 (both directions): optical depth per position and its forward
// exclusive segmented prefix P (carry_P continues a long ray's piece).
template <class SM>
__device__ __forceinline__ void depth_pass(SM& s, const Stage& st, int p0, const SegView& sv, float carry_P,
                                           float tau[8], float P[8], float& incl_end) {
    float a[8], b[8], g[8];
    ld8(st.t0, p0, a);
    ld8(st.t1, p0, b);
    ld8(st.sg, p0, g);
    Seg<1> agg = seg_zero<1>(-1);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        tau[j] = (sv.valid & (1u << j)) ? __fmul_rn(g[j], __fsub_rn(b[j], a[j])) : 0.0f;
        if (sv.head & sv.valid & (1u << j)) agg = seg_zero<1>(0);
        agg.v[0] = agg.v[0] + tau[j];
    }
    Seg<1> cin;
    cin.v[0] = carry_P;
    cin.id = 0;
    const Seg<1> ex = comb(cin, block_scan<1, true>(s, agg, 0));
    float run = ex.v[0];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (sv.head & sv.valid & (1u << j)) run = 0.0f;
        P[j] = run;
        run = run + tau[j];
    }
    incl_end = run;
}

// Forward compositing of a tile of whole rays.
template <class SM>
__device__ void fwd_tile(const RArgs& A, SM& s, Stage& st) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int p0 = tid * kItems;
    const int o_rel = (int)(st.d.base - st.d.abase);
    const int pend = o_rel + st.d.n;
    const long long r0 = st.d.r0;
    const SegView sv = seg_view(st.seg, p0, o_rel, pend);
    float tau[8], P[8], incl_end;
    depth_pass(s, st, p0, sv, 0.0f, tau, P, incl_end);

    float a[8], b[8], c[24], w[8];
    ld8(st.t0, p0, a);
    ld8(st.t1, p0, b);
    ld24(st.c, p0, c);
    float loc[6] = {0, 0, 0, 0, 0, 0};    // sums since the last head (or the thread start)
    float first[6] = {0, 0, 0, 0, 0, 0};  // sums of the items before the first head
    bool seen_head = false;
    bool open_last = false;  // the last segment started here and continues past the thread
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        w[j] = 0.0f;
        if (!(sv.valid & (1u << j))) continue;
        if (sv.head & (1u << j)) {
            if (!seen_head) {
#pragma unroll
                for (int k = 0; k < 6; ++k) first[k] = loc[k];
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) loc[k] = 0.0f;
            seen_head = true;
        }
        const bool kept = !(P[j] > A.thr);
        w[j] = kept ? __expf(-P[j]) * one_minus_exp_neg(tau[j]) : 0.0f;
        const float m = 0.5f * (a[j] + b[j]);
        loc[0] += w[j] * c[3 * j + 0];
        loc[1] += w[j] * c[3 * j + 1];
        loc[2] += w[j] * c[3 * j + 2];
        loc[3] += w[j];
        loc[4] += w[j] * m;
        loc[5] += kept ? tau[j] : 0.0f;
        open_last = seen_head;
        if (sv.tail & (1u << j)) {
            open_last = false;
            if (seen_head) write_ray(A, r0 + tail_id(sv, j), loc);  // started and ended in this thread
        }
    }
    if (!seen_head) {
#pragma unroll
        for (int k = 0; k < 6; ++k) first[k] = loc[k];
    }
    if (A.w_out) st8_global(A.w_out, st.d.abase, p0, sv.valid, w);
    // park the partial sums in this thread's own slots of the spent t0 / t1 planes
    float* pf = &st.t0[p0];
    float* pl = &st.t1[p0];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        pf[k] = first[k];
        pl[k] = open_last ? loc[k] : 0.0f;
    }
    consumer_sync();
    // one warp per ray that spans threads: last part of the head thread plus the
    // first parts of the following threads up to the tail thread
    const int e = st.d.e;
    for (int k = wid; k < e; k += kConsumerWarps) {
        const int h = st.d.off_rel[k], t = st.d.off_rel[k + 1] - 1;
        if (t < h) continue;  // empty ray
        const int th = h >> 3, tt = t >> 3;
        if (th == tt) continue;  // finished by its thread
        float v[6] = {0, 0, 0, 0, 0, 0};
        for (int q = lane; q <= tt - th; q += 32) {
            const float* src = q == 0 ? &st.t1[th * kItems] : &st.t0[(th + q) * kItems];
#pragma unroll
            for (int kk = 0; kk < 6; ++kk) v[kk] += src[kk];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int kk = 0; kk < 6; ++kk) v[kk] += __shfl_xor_sync(0xffffffffu, v[kk], o);
        if (lane == 0) write_ray(A, r0 + k, v);
    }
}

// One piece of a long ray (carried scan state).
//   MODE 0: forward (outputs at the ray's end, weights)
//   MODE 1: totals only (first pass of the adjoint)
//   MODE 2: adjoint with suffix = total - inclusive prefix
template <int MODE, class SM>
__device__ __noinline__ void long_piece(const RArgs& A, SM& s, Stage& st, const float* pray, Carry& carry, const float* tot) {
    const int tid = threadIdx.x;
    const int p0 = tid * kItems;
    const int o_rel = (int)(st.d.base - st.d.abase);
    const int pend = o_rel + st.d.n;
    const long long ray = st.d.r0;
    const SegView sv = seg_view(st.seg, p0, o_rel, pend);
    float tau[8], P[8], incl_end;
    depth_pass(s, st, p0, sv, carry.P, tau, P, incl_end);
    if (tid == (pend - 1) / kItems) s.carry[0] = incl_end;
    float a[8], b[8], c[24], w[8];
    ld8(st.t0, p0, a);
    ld8(st.t1, p0, b);
    ld24(st.c, p0, c);
    Seg<6> loc = seg_zero<6>(-1);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        w[j] = 0.0f;
        if (!(sv.valid & (1u << j))) continue;
        if (sv.head & (1u << j)) loc = seg_zero<6>(0);
        const bool kept = !(P[j] > A.thr);
        w[j] = kept ? __expf(-P[j]) * one_minus_exp_neg(tau[j]) : 0.0f;
        const float m = 0.5f * (a[j] + b[j]);
        loc.v[0] += w[j] * c[3 * j + 0];
        loc.v[1] += w[j] * c[3 * j + 1];
        loc.v[2] += w[j] * c[3 * j + 2];
        loc.v[3] += w[j];
        loc.v[4] += w[j] * m;
        loc.v[5] += kept ? tau[j] : 0.0f;
    }
    if (MODE == 0 && A.w_out) st8_global(A.w_out, st.d.abase, p0, sv.valid, w);
    Seg<6> cin6;
#pragma unroll
    for (int k = 0; k < 6; ++k) cin6.v[k] = carry.acc[k];
    cin6.id = 0;
    const Seg<6> ex = comb(cin6, block_scan<6, true>(s, loc, 1));
    const Seg<6> fin = comb(ex, loc);  // inclusive sums at this thread's last item
    if (MODE == 0 && (sv.tail & sv.valid)) write_ray(A, ray, fin.v);
    if (MODE == 2) {
        const float gC0 = pray[0], gC1 = pray[1], gC2 = pray[2], gA = pray[3], gD = pray[4];
        const float TNtot = __expf(-tot[5]);
        float run[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) run[k] = ex.v[k];
        float gs[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            gs[j] = 0.0f;
            if (!(sv.valid & (1u << j))) continue;
            if (sv.head & (1u << j)) {
#pragma unroll
                for (int k = 0; k < 6; ++k) run[k] = 0.0f;
            }
            const float cr = c[3 * j], cg = c[3 * j + 1], cb = c[3 * j + 2];
            const float m = 0.5f * (a[j] + b[j]);
            run[0] += w[j] * cr;
            run[1] += w[j] * cg;
            run[2] += w[j] * cb;
            run[4] += w[j] * m;
            const bool kept = !(P[j] > A.thr);
            float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
            if (kept) {
                const float Tn = __expf(-(P[j] + tau[j]));
                const float dt = __fsub_rn(b[j], a[j]);
                const float g = gC0 * (Tn * cr - (tot[0] - run[0]) - TNtot * A.bg0) +
                                gC1 * (Tn * cg - (tot[1] - run[1]) - TNtot * A.bg1) +
                                gC2 * (Tn * cb - (tot[2] - run[2]) - TNtot * A.bg2) + gA * TNtot +
                                gD * (Tn * m - (tot[4] - run[4]));
                gs[j] = dt * g;
                g0 = w[j] * gC0;
                g1 = w[j] * gC1;
                g2 = w[j] * gC2;
            }
            c[3 * j + 0] = g0;
            c[3 * j + 1] = g1;
            c[3 * j + 2] = g2;
        }
        st8_global(A.g_sg, st.d.abase, p0, sv.valid, gs);
        st24_global(A.g_c, st.d.abase, p0, sv.valid, c);
    }
    // carry to the next piece: the inclusive sums at the piece's last position
    if (tid == (pend - 1) / kItems) {
#pragma unroll
        for (int k = 0; k < 6; ++k) s.carry[1 + k] = fin.v[k];
    }
    consumer_sync();
    carry.P = s.carry[0];
#pragma unroll
    for (int k = 0; k < 6; ++k) carry.acc[k] = s.carry[1 + k];
    consumer_sync();  // s.carry is rewritten by the next piece
}

// Adjoint of a tile of whole rays: forward scan for T, reverse segmented scan
// for the suffix sums (with the local id of the segment's tail copied along).
template <class SM>
__device__ void bwd_tile(const RArgs& A, SM& s, Stage& st, const float* pray) {
    const int tid = threadIdx.x;
    const int p0 = tid * kItems;
    const int o_rel = (int)(st.d.base - st.d.abase);
    const int pend = o_rel + st.d.n;
    const SegView sv = seg_view(st.seg, p0, o_rel, pend);
    float tau[8], P[8], incl_end;
    depth_pass(s, st, p0, sv, 0.0f, tau, P, incl_end);

    float a[8], b[8], c[24];
    ld8(st.t0, p0, a);
    ld8(st.t1, p0, b);
    ld24(st.c, p0, c);
    float w[8];
    Seg<5> agg = seg_zero<5>(-1);
#pragma unroll
    for (int j = 7; j >= 0; --j) {
        w[j] = 0.0f;
        if (!(sv.valid & (1u << j))) continue;
        if (sv.tail & (1u << j)) agg = seg_zero<5>(tail_id(sv, j));
        const bool kept = !(P[j] > A.thr);
        w[j] = kept ? __expf(-P[j]) * one_minus_exp_neg(tau[j]) : 0.0f;
        const float m = 0.5f * (a[j] + b[j]);
        agg.v[0] += w[j] * c[3 * j + 0];
        agg.v[1] += w[j] * c[3 * j + 1];
        agg.v[2] += w[j] * c[3 * j + 2];
        agg.v[3] += w[j] * m;
        agg.v[4] += kept ? tau[j] : 0.0f;
    }
    Seg<5> run = block_scan<5, false>(s, agg, 1);
    ld8(st.t0, p0, a);
    ld8(st.t1, p0, b);
    ld24(st.c, p0, c);
    float gs[8];
#pragma unroll
    for (int j = 7; j >= 0; --j) {
        gs[j] = 0.0f;
        if (!(sv.valid & (1u << j))) {
            c[3 * j] = c[3 * j + 1] = c[3 * j + 2] = 0.0f;
            continue;
        }
        if (sv.tail & (1u << j)) run = seg_zero<5>(tail_id(sv, j));
        const float cr = c[3 * j], cg = c[3 * j + 1], cb = c[3 * j + 2];
        const float m = 0.5f * (a[j] + b[j]);
        const bool kept = !(P[j] > A.thr);
        float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
        if (kept) {
            const float* pr = &pray[5 * run.id];
            const float gC0 = pr[0], gC1 = pr[1], gC2 = pr[2], gA = pr[3], gD = pr[4];
            const float incl = P[j] + tau[j];
            const float Tn = __expf(-incl);
            const float TN = __expf(-(incl + run.v[4]));
            const float dt = __fsub_rn(b[j], a[j]);
            const float g = gC0 * (Tn * cr - run.v[0] - TN * A.bg0) + gC1 * (Tn * cg - run.v[1] - TN * A.bg1) +
                            gC2 * (Tn * cb - run.v[2] - TN * A.bg2) + gA * TN + gD * (Tn * m - run.v[3]);
            gs[j] = dt * g;
            g0 = w[j] * gC0;
            g1 = w[j] * gC1;
            g2 = w[j] * gC2;
        }
        run.v[0] += w[j] * cr;
        run.v[1] += w[j] * cg;
        run.v[2] += w[j] * cb;
        run.v[3] += w[j] * m;
        run.v[4] += kept ? tau[j] : 0.0f;
        c[3 * j + 0] = g0;
        c[3 * j + 1] = g1;
        c[3 * j + 2] = g2;
    }
    st8_global(A.g_sg, st.d.abase, p0, sv.valid, gs);
    st24_global(A.g_c, st.d.abase, p0, sv.valid, c);
}

template <bool kBwd>
__device__ void consume(const RArgs& A, Smem<kBwd>& s) {
    const int tid = threadIdx.x;
    Carry carry;
    carry.P = 0.0f;
#pragma unroll
    for (int k = 0; k < 6; ++k) carry.acc[k] = 0.0f;
    float tot[6] = {0, 0, 0, 0, 0, 0};
    for (int it = 0;; ++it) {
        const int stg = it % kStages;
        const uint32_t ph = (uint32_t)(it / kStages) & 1u;
        const bool got = mbar_wait_bounded(&s.full[stg], ph, kWaitLimitNs);
        if (!consumer_all(got)) {
            if (tid == 0) report_timeout();
            return;
        }
        Stage& st = s.st[stg];
        const float* pray = kBwd ? s.pray[stg] : nullptr;
        const int kind = st.d.kind;
        if (kind == kKindDone) return;
        if (st.d.cend < st.d.base + st.d.n) {  // the arrays' last samples: plain loads
            load_ragged_end(A, st);
            consumer_sync();
        }
        if (kind == kKindTile) {
            if (!kBwd && tid < st.d.e && st.d.off_rel[tid + 1] == st.d.off_rel[tid]) {
                const long long ray = st.d.r0 + tid;  // empty ray
                A.rgb_out[3 * ray + 0] = A.bg0;
                A.rgb_out[3 * ray + 1] = A.bg1;
                A.rgb_out[3 * ray + 2] = A.bg2;
                A.op_out[ray] = 0.0f;
                A.dep_out[ray] = 0.0f;
                A.tr_out[ray] = 1.0f;
            }
            if (st.d.n > 0) {
                if (!kBwd)
                    fwd_tile(A, s, st);
                else
                    bwd_tile(A, s, st, pray);
            }
        } else {  // one piece of a long ray (local id 0)
            const int flags = st.d.flags;
            if (flags & kFirst) {
                carry.P = 0.0f;
#pragma unroll
                for (int k = 0; k < 6; ++k) carry.acc[k] = 0.0f;
            }
            if (!kBwd) {
                long_piece<0>(A, s, st, pray, carry, nullptr);
            } else if (!(flags & kPass2)) {
                long_piece<1>(A, s, st, pray, carry, nullptr);
                if (flags & kLast) {
#pragma unroll
                    for (int k = 0; k < 6; ++k) tot[k] = carry.acc[k];
                }
            } else {
                long_piece<2>(A, s, st, pray, carry, tot);
            }
        }
        // each warp releases the stage once it is done with it
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&s.empty[stg]);
    }
}

// 8 warps x 128 registers: two CTAs (16 warps, 4 per scheduler) resident per SM.
template <bool kBwd>
__global__ void __maxnreg__(128) k_render(RArgs A) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem<kBwd>& s = *reinterpret_cast<Smem<kBwd>*>(smem_raw);
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&s.full[i], 1);
            mbar_init(&s.empty[i], kConsumerWarps);
        }
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x >= kConsumers) {
        const int64_t S = __ldg(&A.off[A.n_rays]);
        const int64_t nchunks = S / kChunk + 1;
        const int64_t per = (nchunks + gridDim.x - 1) / gridDim.x;
        const int64_t cb = min64((int64_t)blockIdx.x * per, nchunks);
        const int64_t ce = min64(cb + per, nchunks);
        Producer<kBwd> pr{A, s, (long long)(S & ~3ll), 0, true};
        pr.run(cb, ce);
    } else {
        consume<kBwd>(A, s);
    }
}

// A wait on an mbarrier that nothing arrives on: exercises the bounded-wait
// path (timeout -> status word) without disturbing the GPU.
__global__ void k_selftest_wait(uint64_t limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
    if (!ok && threadIdx.x == 0) report_timeout();
}

template <bool kBwd>
int launch_render_t(const RArgs& A, cudaStream_t st) {
    const size_t smem = sizeof(Smem<kBwd>);
    int per_sm = 1;
    NACC_CUDA_TRY(cudaFuncSetAttribute(k_render<kBwd>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    NACC_CUDA_TRY(cudaFuncSetAttribute(k_render<kBwd>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared));
    NACC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render<kBwd>, kThreads, smem));
    if (per_sm < 1) per_sm = 1;
    k_render<kBwd><<<per_sm * sm_count(), kThreads, smem, st>>>(A);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

int check_common(int64_t n_rays, const int64_t* offsets, const float* t_starts, const float* t_ends,
                 const float* sigmas, const float* rgbs, const float* bg) {
    NACC_CHECK_ARG(n_rays >= 0 && n_rays < (int64_t(1) << 40), "n_rays=%lld out of range", (long long)n_rays);
    NACC_CHECK_ARG(offsets != nullptr, "offsets is NULL");
    NACC_CHECK_ARG(bg != nullptr, "bg is NULL");
    NACC_CHECK_ARG(t_starts && t_ends && sigmas && rgbs, "a sample array is NULL");
    NACC_CHECK_ARG(aligned16(t_starts) && aligned16(t_ends) && aligned16(sigmas) && aligned16(rgbs),
                   "t_starts, t_ends, sigmas and rgbs must be 16-byte aligned");
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
    NACC_CHECK_ARG(weights_out == nullptr || aligned16(weights_out), "weights_out must be 16-byte aligned");
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
    return launch_render_t<false>(A, as_stream(stream));
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
    NACC_CHECK_ARG(aligned16(g_sigmas) && aligned16(g_rgbs), "g_sigmas and g_rgbs must be 16-byte aligned");
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
    return launch_render_t<true>(A, as_stream(stream));
}

extern "C" int nacc_device_status(void* stream, int32_t* status_out) {
    clear_error();
    NACC_CHECK_ARG(status_out != nullptr, "status_out is NULL");
    unsigned int v = 0;
    NACC_CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
    NACC_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_nacc_render_status, sizeof(v)));
    const unsigned int zero = 0;
    NACC_CUDA_TRY(cudaMemcpyToSymbol(g_nacc_render_status, &zero, sizeof(zero)));
    *status_out = (v & 1u) ? NACC_ERR_TIMEOUT : NACC_OK;
    return NACC_OK;
}

extern "C" int nacc_selftest_wait_timeout(int64_t limit_ns, void* stream) {
    clear_error();
    NACC_CHECK_ARG(limit_ns > 0 && limit_ns <= 100000000, "limit_ns must be in (0, 1e8]");
    k_selftest_wait<<<1, 32, 0, as_stream(stream)>>>((uint64_t)limit_ns);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}
