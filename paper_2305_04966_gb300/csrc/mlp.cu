// mlp.cu -- the learned density proposal (nacc_proposal.h): frequency
// encoding and a 3-layer width-64 MLP whose two 64x64 layers run on the
// tcgen05 tensor cores (BF16 operands in shared memory, FP32 accumulators in
// tensor memory), plus its fused adjoint and Adam.
//
// Table 1 "PDF Approaches" and Sec. 3.2 of NerfAcc (arXiv 2305.04966): a
// small network predicts density; its transmittance gives the PDF that
// inverse transform sampling (Eq. 1) resamples.
//
// Forward (persistent CTAs of 128 threads, 128 points per tile, thread t =
// point t of the tile): the thread encodes its point into row t of a
// K-major, 128-byte-swizzled BF16 tile; one thread issues the four
// K = 16 MMAs of a layer (M = 128 points, N = 64 units, K = 64); every warp
// reads its 32 rows of the accumulator back from tensor memory, applies ReLU
// while packing the next layer's BF16 input row (layer 1's bias rides in the
// MMA through the encoding's padding columns); layer 2's output gets b2, ReLU
// and BF16 rounding and goes straight into the last layer (64 -> 1) as FP32
// FMAs on the CUDA cores, then b3 and softplus.
//
// Adjoint (same tiles): delta3 = dL/dz3, delta2 = delta3 w3 * [h2 > 0] and
// delta1 = (delta2 W2) * [h1 > 0] (an M = 128 MMA against W2^T); the weight
// gradients dW2 = delta2^T h1 and dW1 = delta1^T e are M = 64 MMAs with K =
// the 128 points of the tile, accumulated in tensor memory over all tiles of
// the CTA (their operands are written transposed into shared memory, so
// every MMA uses the same K-major layout).  Bias and w3 gradients are column
// sums on the CUDA cores.  Waits on MMA completion are bounded (2 s).
#include <cuda_bf16.h>

#include "../../include/nacc_proposal.h"
#include "nacc_internal.cuh"
#include "tcgen05.cuh"

// bit 0: a bounded wait expired in a proposal-network kernel
__device__ unsigned int g_nacc_mlp_status;

namespace nacc {
namespace {

constexpr int kTile = 128;
constexpr int kThreads = 128;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int oW1 = 0, oB1 = 4096, oW2 = 4160, oB2 = 8256, oW3 = 8320, oB3 = 8384;
constexpr int wW1 = 0, wW2 = 4096, wW3 = 8192;
constexpr uint32_t kTileBytes = 16384;  // 128 rows x 128 bytes
constexpr uint32_t kWBytes = 8192;      // 64 rows x 128 bytes

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
    return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// e(x): [x, y, z, (sin, cos)(2^k pi x_a) for k = 0..7, a = 0..2], padded to 64
// with `pad` in columns 51 and 52 (0; the forward kernel puts ones there,
// which carry layer 1's bias) and zeros after.  Half H of the row (columns
// 32H .. 32H+31) needs the bands k = 0..4 (H = 0) or 4..7 (H = 1).  The
// even bands of each half are evaluated directly: sin(2^k pi x) = sin(2 pi f)
// with f the phase 2^(k-1) x reduced exactly to [-1/2, 1/2] (power-of-two
// scaling and u - rint(u) are exact in FP32), then the hardware sine and
// cosine of 2 pi f (|2 pi f| <= pi: absolute error below 4.3e-7).  The odd
// bands come from the band below by the double-angle identities sin 2a =
// 2 sin a cos a, cos 2a = (cos a - sin a)(cos a + sin a), which at most
// double that error and add a few roundings: below 1.3e-6 in every column.
template <int H>
__device__ __forceinline__ void encode_half(float x, float y, float z, float e[32], float pad = 0.0f) {
    constexpr int k0 = H == 0 ? 0 : 4, k1 = H == 0 ? 4 : 7;
    const float c[3] = {x, y, z};
    float sn[8][3], cs[8][3];
#pragma unroll
    for (int k = k0; k <= k1; ++k) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (((k - k0) & 1) == 0) {
                const float u = c[a] * (0.5f * (float)(1 << k));
                const float f = u - rintf(u);
                __sincosf(6.28318531f * f, &sn[k][a], &cs[k][a]);
            } else {
                const float s0 = sn[k - 1][a], c0 = cs[k - 1][a];
                sn[k][a] = (s0 + s0) * c0;
                cs[k][a] = (c0 - s0) * (c0 + s0);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const int col = 32 * H + i;
        if (col < 3) {
            e[i] = c[col];
        } else if (col < 51) {
            const int q = col - 3, k = q / 6, a = (q % 6) / 2;
            e[i] = (q & 1) ? cs[k][a] : sn[k][a];
        } else {
            e[i] = col < 53 ? pad : 0.0f;
        }
    }
}

__device__ __forceinline__ void encode_point(float x, float y, float z, float e[64], float pad51 = 0.0f) {
    encode_half<0>(x, y, z, e, pad51);
    encode_half<1>(x, y, z, e + 32, pad51);
}

// Two FP32 values -> BF16x2 (round to nearest even) with ReLU: lo in the low half.
__device__ __forceinline__ uint32_t pack_relu_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// Row r (64 values -> BF16) of a K-major SW128 tile.
__device__ __forceinline__ void store_row(uint8_t* tile, int r, const float v[64]) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        uint4 q;
        q.x = pack_bf16x2(v[8 * c + 0], v[8 * c + 1]);
        q.y = pack_bf16x2(v[8 * c + 2], v[8 * c + 3]);
        q.z = pack_bf16x2(v[8 * c + 4], v[8 * c + 5]);
        q.w = pack_bf16x2(v[8 * c + 6], v[8 * c + 7]);
        *reinterpret_cast<uint4*>(tile + (r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4)) = q;
    }
}

// Column p (64 values, one per row) of a [64 rows][128 K] tile made of two
// K-major SW128 sub-tiles of 64 K each (the transposed operands).
__device__ __forceinline__ void store_col(uint8_t* tile2, int p, const float v[64]) {
    uint8_t* sub = tile2 + (p >> 6) * kWBytes;
#pragma unroll
    for (int i = 0; i < 64; ++i)
        *reinterpret_cast<__nv_bfloat16*>(sub + tc::sw128_offset(i, p & 63)) = __float2bfloat16_rn(v[i]);
}

// A value as the sum of two BF16 numbers: hi = bf16(v), lo = bf16(v - hi)
// (v - hi is exact in FP32), within 2^-18 |v| of v.  The training kernel's
// error terms go to the tensor cores as both parts, so its products carry
// about 16 significant bits of the FP32 terms instead of 8.
__device__ __forceinline__ float bf16_lo(float v) { return v - __bfloat162float(__float2bfloat16_rn(v)); }

// Row r of the heads and of the tails of v into two K-major SW128 tiles.
__device__ __forceinline__ void store_row_split(uint8_t* tile_hi, uint8_t* tile_lo, int r, const float v[64]) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        uint4 q, w;
        q.x = pack_bf16x2(v[8 * c + 0], v[8 * c + 1]);
        q.y = pack_bf16x2(v[8 * c + 2], v[8 * c + 3]);
        q.z = pack_bf16x2(v[8 * c + 4], v[8 * c + 5]);
        q.w = pack_bf16x2(v[8 * c + 6], v[8 * c + 7]);
        w.x = pack_bf16x2(bf16_lo(v[8 * c + 0]), bf16_lo(v[8 * c + 1]));
        w.y = pack_bf16x2(bf16_lo(v[8 * c + 2]), bf16_lo(v[8 * c + 3]));
        w.z = pack_bf16x2(bf16_lo(v[8 * c + 4]), bf16_lo(v[8 * c + 5]));
        w.w = pack_bf16x2(bf16_lo(v[8 * c + 6]), bf16_lo(v[8 * c + 7]));
        const uint32_t off = (r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4);
        *reinterpret_cast<uint4*>(tile_hi + off) = q;
        *reinterpret_cast<uint4*>(tile_lo + off) = w;
    }
}

// Column p of the heads and of the tails (see store_col).
__device__ __forceinline__ void store_col_split(uint8_t* tile2_hi, uint8_t* tile2_lo, int p, const float v[64]) {
    const uint32_t sub = (p >> 6) * kWBytes;
#pragma unroll
    for (int i = 0; i < 64; ++i) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v[i]);
        const uint32_t off = sub + tc::sw128_offset(i, p & 63);
        *reinterpret_cast<__nv_bfloat16*>(tile2_hi + off) = h;
        *reinterpret_cast<__nv_bfloat16*>(tile2_lo + off) = __float2bfloat16_rn(v[i] - __bfloat162float(h));
    }
}

__device__ __forceinline__ float load_elem(const uint8_t* tile, int r, int k) {
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(tile + tc::sw128_offset(r, k)));
}

// Accumulator row (this thread's lane) of a 128 x 64 FP32 tile in tensor memory.
__device__ __forceinline__ void tmem_row64(uint32_t taddr, float v[64]) {
    tc::tmem_ld16(taddr, v);
    tc::tmem_ld16(taddr + 16, v + 16);
    tc::tmem_ld16(taddr + 32, v + 32);
    tc::tmem_ld16(taddr + 48, v + 48);
    tc::tmem_wait_ld();
}

// Make this thread's shared-memory writes visible to the tensor cores and
// order them (and earlier tensor-memory reads) before the MMA issue.
__device__ __forceinline__ void sync_for_mma() {
    fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// Thread 0 waits (bounded) for the MMA completion; the others wait at the
// CTA barrier instead of polling, then order their tensor-memory reads after it.
__device__ __forceinline__ bool wait_mma(uint64_t* bar, uint32_t& phase) {
    const bool mine = threadIdx.x == 0 ? mbar_wait_bounded(bar, phase & 1u, kWaitNs) : true;
    const bool ok = __syncthreads_and(mine);
    ++phase;
    tc::fence_after_sync();
    return ok;
}

__device__ __forceinline__ float softplus(float z) { return z > 20.0f ? z : log1pf(expf(z)); }

__device__ __forceinline__ void load_weight_tile(uint8_t* dst, const uint16_t* w, bool transpose) {
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) {
        const int a = i >> 6, b = i & 63;  // w[a][b]
        const int r = transpose ? b : a, k = transpose ? a : b;
        *reinterpret_cast<uint16_t*>(dst + tc::sw128_offset(r, k)) = w[i];
    }
}

// Where the points come from: an array xyz [n][3], or the midpoints of the
// bins of rays (point p = bin p % nb of ray p / nb, x = o + t d with t the
// midpoint of edges [ray][bin], [ray][bin + 1]).
struct PointSrc {
    const float* xyz;
    const float* o;
    const float* d;
    const float* edges;
    int nb;
    int contract;  // rays: feed c(x), the L-infinity contraction of the bin midpoint
    int p32;       // rays: n_rays * nb < 2^32
    const uint16_t* enc = nullptr;  // rows already encoded (BF16, [n][64]): replaces the encoding
};

// Row p of an encoded input (64 BF16 values, 16-byte aligned rows).
__device__ __forceinline__ void load_enc_row(const uint16_t* enc, int64_t p, float v[64]) {
    const uint4* q = reinterpret_cast<const uint4*>(enc + 64 * p);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint4 w = q[c];
        const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[8 * c + 2 * k] = __uint_as_float(u[k] << 16);
            v[8 * c + 2 * k + 1] = __uint_as_float(u[k] & 0xffff0000u);
        }
    }
}

__device__ __forceinline__ void point_of(const PointSrc& S, int64_t p, float& x, float& y, float& z) {
    if (S.xyz) {
        x = S.xyz[3 * p];
        y = S.xyz[3 * p + 1];
        z = S.xyz[3 * p + 2];
        return;
    }
    int64_t r, b;
    if (S.p32) {  // every point index fits 32 bits: the cheaper division
        const uint32_t q = (uint32_t)p / (uint32_t)S.nb;
        r = q;
        b = (uint32_t)p - q * (uint32_t)S.nb;
    } else {
        r = p / S.nb;
        b = p - r * S.nb;
    }
    const float* e = S.edges + r * (S.nb + 1) + b;
    const float t = 0.5f * (e[0] + e[1]);
    x = fmaf(S.d[3 * r], t, S.o[3 * r]);
    y = fmaf(S.d[3 * r + 1], t, S.o[3 * r + 1]);
    z = fmaf(S.d[3 * r + 2], t, S.o[3 * r + 2]);
    if (S.contract) {
        const float m = fmaxf(fmaxf(fabsf(x), fabsf(y)), fabsf(z));
        if (m > 1.0f) {  // x (2 - 1/m) / m
            const float inv = __fdiv_rn(1.0f, m);
            const float g = __fmul_rn(__fsub_rn(2.0f, inv), inv);
            x = __fmul_rn(x, g);
            y = __fmul_rn(y, g);
            z = __fmul_rn(z, g);
        }
    }
}

// Layer 1's weight tile with its bias in the encoding's padding columns 51
// and 52 (which the forward kernel sets to one): b1 = hi + lo, hi = bf16(b1),
// lo = bf16(b1 - hi) (b1 to about 2^-17 relative; the definition's padding
// weights multiply zeros, so replacing them changes nothing else).
__device__ __forceinline__ void load_w1_bias_tile(uint8_t* dst, const uint16_t* w, const float* P) {
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) {
        const int a = i >> 6, b = i & 63;
        uint16_t v = w[i];
        if (b == 51 || b == 52) {
            const float b1 = P[oB1 + a];
            const __nv_bfloat16 hi = __float2bfloat16_rn(b1);
            const __nv_bfloat16 h = b == 51 ? hi : __float2bfloat16_rn(b1 - __bfloat162float(hi));
            v = *reinterpret_cast<const uint16_t*>(&h);
        }
        *reinterpret_cast<uint16_t*>(dst + tc::sw128_offset(a, b)) = v;
    }
}

// 32 accumulator columns (this thread's row) -> + bias (or none) -> ReLU ->
// BF16, into 16-byte chunks c0, c0+1, c0+2, c0+3 of row r of a SW128 tile.
__device__ __forceinline__ void relu_pack32(uint32_t taddr, const float* bias, uint8_t* tile, int r, int c0) {
    float v[32];
    tc::tmem_ld16(taddr, v);
    tc::tmem_ld16(taddr + 16, v + 16);
    tc::tmem_wait_ld();
    if (bias) {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] += bias[i];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint4 q;
        q.x = pack_relu_bf16x2(v[8 * c + 0], v[8 * c + 1]);
        q.y = pack_relu_bf16x2(v[8 * c + 2], v[8 * c + 3]);
        q.z = pack_relu_bf16x2(v[8 * c + 4], v[8 * c + 5]);
        q.w = pack_relu_bf16x2(v[8 * c + 6], v[8 * c + 7]);
        *reinterpret_cast<uint4*>(tile + (r >> 3) * 1024 + (r & 7) * 128 + (((c0 + c) ^ (r & 7)) << 4)) = q;
    }
}

// z3 += sum over 32 accumulator columns (this thread's row) of
// bf16(relu(acc + b2)) * w3, in column order (FP32 FMAs).
__device__ __forceinline__ float head_dot32(uint32_t taddr, const float* b2, const float* w3, float z) {
    float v[32];
    tc::tmem_ld16(taddr, v);
    tc::tmem_ld16(taddr + 16, v + 16);
    tc::tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 32; i += 2) {
        const uint32_t h = pack_relu_bf16x2(v[i] + b2[i], v[i + 1] + b2[i + 1]);
        z = fmaf(__uint_as_float(h << 16), w3[i], z);
        z = fmaf(__uint_as_float(h & 0xffff0000u), w3[i + 1], z);
    }
    return z;
}

// Forward.  Per tile: encode -> MMA (layer 1, bias folded) -> ReLU/BF16 ->
// MMA (layer 2) -> + b2, ReLU/BF16 and the 64 -> 1 head on the CUDA cores
// (FP32 FMAs in column order) -> + b3, softplus.
template <bool kEnc>  // kEnc: the rows come encoded (S.enc)
__global__ void __launch_bounds__(kThreads) k_mlp_forward(int64_t n, PointSrc S, const float* __restrict__ P,
                                                          const uint16_t* __restrict__ Wb,
                                                          float* __restrict__ sigma) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = align1024(smem_raw);
    uint8_t* sW1 = base;
    uint8_t* sW2 = base + kWBytes;
    uint8_t* sX = base + 2 * kWBytes;
    __shared__ float sB2[64];
    __shared__ float sW3[64];
    __shared__ float sB3;
    __shared__ uint64_t bar;
    __shared__ uint32_t tbase;
    const int t = threadIdx.x, warp = t >> 5;
    load_w1_bias_tile(sW1, Wb + wW1, P);
    load_weight_tile(sW2, Wb + wW2, false);
    if (t < 64) {
        sB2[t] = P[oB2 + t];
        sW3[t] = __uint_as_float((uint32_t)Wb[wW3 + t] << 16);  // the BF16 w3
    }
    if (t == 0) {
        sB3 = P[oB3];
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(&tbase, 64);
        tc::tmem_relinquish();
    }
    sync_for_mma();
    const uint32_t tm = tbase, row = tm + ((uint32_t)(warp * 32) << 16);
    const uint32_t idesc = tc::idesc_bf16_f32(128, 64);
    const uint64_t dX = tc::sw128_desc(smem_u32(sX)), dW1 = tc::sw128_desc(smem_u32(sW1)),
                   dW2 = tc::sw128_desc(smem_u32(sW2));
    uint32_t phase = 0;
    bool ok = true;
    const int64_t ntiles = (n + kTile - 1) / kTile;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t p = tile * kTile + t;
        {
            float v[64];
            if (kEnc && p < n) {  // the padding columns 51 and 52 carry the folded bias
                load_enc_row(S.enc, p, v);
                v[51] = 1.0f;
                v[52] = 1.0f;
            } else if (p < n) {
                float x, y, z;
                point_of(S, p, x, y, z);
                encode_point(x, y, z, v, 1.0f);
            } else {
#pragma unroll
                for (int i = 0; i < 64; ++i) v[i] = 0.0f;
            }
            store_row(sX, t, v);
        }
        sync_for_mma();
        if (t == 0) {
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) tc::mma_bf16(tm, dX + 2 * ks, dW1 + 2 * ks, idesc, ks > 0);
            tc::mma_commit(&bar);
        }
        if (!(ok = wait_mma(&bar, phase))) break;
        relu_pack32(row, nullptr, sX, t, 0);
        relu_pack32(row + 32, nullptr, sX, t, 4);
        sync_for_mma();
        if (t == 0) {
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) tc::mma_bf16(tm, dX + 2 * ks, dW2 + 2 * ks, idesc, ks > 0);
            tc::mma_commit(&bar);
        }
        if (!(ok = wait_mma(&bar, phase))) break;
        float z = head_dot32(row, sB2, sW3, 0.0f);
        z = head_dot32(row + 32, sB2 + 32, sW3 + 32, z);
        if (p < n) sigma[p] = softplus(z + sB3);
        tc::fence_before_sync();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tm, 64);
    if (!ok && t == 0) atomicOr(&g_nacc_mlp_status, 1u);
}

// Shared-memory map of the training kernel (offsets from a 1 KiB-aligned base).
constexpr uint32_t tW1 = 0, tW2 = 8192, tW2T = 16384;       // 64 x 64 weight tiles
constexpr uint32_t tE = 24576;                              // 128 x 64: e, later h2 (point-major)
constexpr uint32_t tET = tE + kTileBytes;                   // 64 x 128: e^T
constexpr uint32_t tH1 = tET + kTileBytes;                  // 128 x 64: h1
constexpr uint32_t tH1T = tH1 + kTileBytes;                 // 64 x 128: h1^T
constexpr uint32_t tD2 = tH1T + kTileBytes;                 // 128 x 64: delta2, later delta1 (heads)
constexpr uint32_t tD2T = tD2 + kTileBytes;                 // 64 x 128: delta2^T (heads)
constexpr uint32_t tD1T = tD2T + kTileBytes;                // 64 x 128: delta1^T (heads)
constexpr uint32_t tD2L = tD1T + kTileBytes;                // the same three for the tails
constexpr uint32_t tD2LT = tD2L + kTileBytes;
constexpr uint32_t tD1LT = tD2LT + kTileBytes;
constexpr uint32_t kTrainSmem = tD1LT + kTileBytes + 1024;  // + alignment slack

__global__ void __launch_bounds__(kThreads, 1)
    k_mlp_train(int64_t n, const float* __restrict__ xyz, const uint16_t* __restrict__ enc,
                const float* __restrict__ target, const float* __restrict__ P, const uint16_t* __restrict__ Wb,
                float* __restrict__ G, float* __restrict__ loss_sum, float two_over_n) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = align1024(smem_raw);
    __shared__ float sB1[64], sB2[64], sW3[64], sD3[kTile];
    __shared__ float sB3;
    __shared__ float sRed[kThreads / 32][2];
    __shared__ uint64_t bar;
    __shared__ uint32_t tbase;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    load_weight_tile(base + tW1, Wb + wW1, false);
    load_weight_tile(base + tW2, Wb + wW2, false);
    load_weight_tile(base + tW2T, Wb + wW2, true);
    if (t < 64) {
        sB1[t] = P[oB1 + t];
        sB2[t] = P[oB2 + t];
        sW3[t] = __bfloat162float(__ushort_as_bfloat16(Wb[wW3 + t]));
    }
    if (t == 0) {
        sB3 = P[oB3];
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(&tbase, 256);  // [0,64) layer outputs, [64,128) delta1, [128,192) dW2, [192,256) dW1
        tc::tmem_relinquish();
    }
    sync_for_mma();
    const uint32_t tm = tbase, row = tm + ((uint32_t)(warp * 32) << 16);
    const uint32_t id128 = tc::idesc_bf16_f32(128, 64), id64 = tc::idesc_bf16_f32(64, 64);
    const uint64_t dE = tc::sw128_desc(smem_u32(base + tE)), dH1 = tc::sw128_desc(smem_u32(base + tH1)),
                   dD2 = tc::sw128_desc(smem_u32(base + tD2)), dD2L = tc::sw128_desc(smem_u32(base + tD2L)),
                   dW1 = tc::sw128_desc(smem_u32(base + tW1)), dW2 = tc::sw128_desc(smem_u32(base + tW2)),
                   dW2T = tc::sw128_desc(smem_u32(base + tW2T));
    const int j = t & 63, half = t >> 6;  // column-sum role: unit j over points [64 half, 64 half + 64)
    float acc_w3 = 0.0f, acc_b2 = 0.0f, acc_b1 = 0.0f, acc_b3 = 0.0f, acc_loss = 0.0f;
    uint32_t phase = 0;
    bool ok = true, first = true;
    const int64_t ntiles = (n + kTile - 1) / kTile;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t p = tile * kTile + t;
        const bool valid = p < n;
        float v[64], h[64];
        if (valid && enc)
            load_enc_row(enc, p, v);
        else if (valid)
            encode_point(xyz[3 * p], xyz[3 * p + 1], xyz[3 * p + 2], v);
        else
#pragma unroll
            for (int i = 0; i < 64; ++i) v[i] = 0.0f;
        store_row(base + tE, t, v);
        store_col(base + tET, t, v);
        sync_for_mma();
        if (t == 0) {  // layer 1
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) tc::mma_bf16(tm, dE + 2 * ks, dW1 + 2 * ks, id128, ks > 0);
            tc::mma_commit(&bar);
        }
        if (!(ok = wait_mma(&bar, phase))) break;
        tmem_row64(row, v);
#pragma unroll
        for (int i = 0; i < 64; ++i) v[i] = fmaxf(v[i] + sB1[i], 0.0f);  // h1
        store_row(base + tH1, t, v);
        store_col(base + tH1T, t, v);
        sync_for_mma();
        if (t == 0) {  // layer 2
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) tc::mma_bf16(tm, dH1 + 2 * ks, dW2 + 2 * ks, id128, ks > 0);
            tc::mma_commit(&bar);
        }
        if (!(ok = wait_mma(&bar, phase))) break;
        tmem_row64(row, v);
        float z = sB3;
#pragma unroll
        for (int i = 0; i < 64; ++i) {
            h[i] = bf16_round(fmaxf(v[i] + sB2[i], 0.0f));  // h2
            z = fmaf(sW3[i], h[i], z);
        }
        float d3 = 0.0f;
        if (valid) {
            const float dd = softplus(z) - target[p];
            acc_loss = fmaf(dd, dd, acc_loss);
            d3 = two_over_n * dd / (1.0f + expf(-z));
        }
        acc_b3 += d3;
        sD3[t] = d3;
        store_row(base + tE, t, h);  // h2 (e's tile is free: layer 1 has completed)
#pragma unroll
        for (int i = 0; i < 64; ++i) v[i] = h[i] > 0.0f ? d3 * sW3[i] : 0.0f;  // delta2
        store_row_split(base + tD2, base + tD2L, t, v);
        store_col_split(base + tD2T, base + tD2LT, t, v);
        sync_for_mma();
        if (t == 0) {
            // delta1 before the mask: delta2 W2  (B = W2^T, K-major over layer-2 units), heads then tails
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) tc::mma_bf16(tm + 64, dD2 + 2 * ks, dW2T + 2 * ks, id128, ks > 0);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) tc::mma_bf16(tm + 64, dD2L + 2 * ks, dW2T + 2 * ks, id128, true);
            // dW2 += delta2^T h1 over the tile's 128 points (M = 64 units, K = points), heads and tails
#pragma unroll
            for (int ks = 0; ks < 16; ++ks) {
                const uint32_t sub = (uint32_t)((ks >> 2) & 1) * kWBytes;
                const uint32_t dt = ks < 8 ? tD2T : tD2LT;
                tc::mma_bf16(tm + 128, tc::sw128_desc(smem_u32(base + dt + sub)) + 2 * (ks & 3),
                             tc::sw128_desc(smem_u32(base + tH1T + sub)) + 2 * (ks & 3), id64, !first || ks > 0);
            }
            tc::mma_commit(&bar);
        }
        // column sums while the tensor cores work: dw3_j = sum delta3 h2_j, db2_j = sum delta2_j
        for (int q = 64 * half; q < 64 * half + 64; ++q) {
            acc_w3 = fmaf(sD3[q], load_elem(base + tE, q, j), acc_w3);
            acc_b2 += load_elem(base + tD2, q, j) + load_elem(base + tD2L, q, j);
        }
        if (!(ok = wait_mma(&bar, phase))) break;
        tmem_row64(row + 64, v);
        const uint8_t* h1row = base + tH1;
#pragma unroll
        for (int i = 0; i < 64; ++i) v[i] = load_elem(h1row, t, i) > 0.0f ? v[i] : 0.0f;  // delta1
        __syncthreads();  // every column-sum read of delta2 is done before delta1 overwrites it
        store_row_split(base + tD2, base + tD2L, t, v);
        store_col_split(base + tD1T, base + tD1LT, t, v);
        sync_for_mma();
        if (t == 0) {  // dW1 += delta1^T e, heads and tails
#pragma unroll
            for (int ks = 0; ks < 16; ++ks) {
                const uint32_t sub = (uint32_t)((ks >> 2) & 1) * kWBytes;
                const uint32_t dt = ks < 8 ? tD1T : tD1LT;
                tc::mma_bf16(tm + 192, tc::sw128_desc(smem_u32(base + dt + sub)) + 2 * (ks & 3),
                             tc::sw128_desc(smem_u32(base + tET + sub)) + 2 * (ks & 3), id64, !first || ks > 0);
            }
            tc::mma_commit(&bar);
        }
        for (int q = 64 * half; q < 64 * half + 64; ++q)
            acc_b1 += load_elem(base + tD2, q, j) + load_elem(base + tD2L, q, j);
        if (!(ok = wait_mma(&bar, phase))) break;
        first = false;
    }
    // weight gradients: M = 64 accumulators, row m in lane (m % 16) + 32 (m / 16)
    if (ok && !first) {  // block-uniform: every lane of each warp takes part in the loads
        const int m = 16 * warp + lane;
        float g[64];
        tmem_row64(row + 128, g);
        if (lane < 16)
            for (int i = 0; i < 64; ++i) atomicAdd(&G[oW2 + 64 * m + i], g[i]);
        tmem_row64(row + 192, g);
        if (lane < 16)
            for (int i = 0; i < 64; ++i) atomicAdd(&G[oW1 + 64 * m + i], g[i]);
    }
    if (ok) {
        atomicAdd(&G[oW3 + j], acc_w3);
        atomicAdd(&G[oB2 + j], acc_b2);
        atomicAdd(&G[oB1 + j], acc_b1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc_b3 += __shfl_xor_sync(0xffffffffu, acc_b3, o);
            acc_loss += __shfl_xor_sync(0xffffffffu, acc_loss, o);
        }
        if (lane == 0) {
            sRed[warp][0] = acc_b3;
            sRed[warp][1] = acc_loss;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (ok && t == 0) {
        float b3 = 0.0f, l = 0.0f;
        for (int w = 0; w < kThreads / 32; ++w) {
            b3 += sRed[w][0];
            l += sRed[w][1];
        }
        atomicAdd(&G[oB3], b3);
        atomicAdd(loss_sum, l);
    }
    if (warp == 0) tc::tmem_dealloc(tm, 256);
    if (!ok && t == 0) atomicOr(&g_nacc_mlp_status, 1u);
}

__global__ void k_mlp_adam(float* __restrict__ P, float* __restrict__ G, float* __restrict__ m,
                           float* __restrict__ v, float lr, float b1, float b2, float eps, float bc1, float bc2,
                           uint16_t* __restrict__ Wb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NACC_MLP_PARAMS; i += gridDim.x * blockDim.x) {
        const float g = G[i];
        const float mi = b1 * m[i] + (1.0f - b1) * g;
        const float vi = b2 * v[i] + (1.0f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float p = P[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        P[i] = p;
        G[i] = 0.0f;
        const uint16_t pb = __bfloat16_as_ushort(__float2bfloat16_rn(p));
        if (i < oB1)
            Wb[wW1 + i] = pb;
        else if (i >= oW2 && i < oB2)
            Wb[wW2 + (i - oW2)] = pb;
        else if (i >= oW3 && i < oB3)
            Wb[wW3 + (i - oW3)] = pb;
    }
}

__global__ void k_mlp_sync(const float* __restrict__ P, uint16_t* __restrict__ Wb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NACC_MLP_WEIGHTS; i += gridDim.x * blockDim.x) {
        const int src = i < wW2 ? oW1 + i : (i < wW3 ? oW2 + (i - wW2) : oW3 + (i - wW3));
        Wb[i] = __bfloat16_as_ushort(__float2bfloat16_rn(P[src]));
    }
}

__global__ void k_mlp_encode(int64_t n, const float* __restrict__ xyz, float* __restrict__ enc) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        float e[64];
        encode_point(xyz[3 * p], xyz[3 * p + 1], xyz[3 * p + 2], e);
        for (int i = 0; i < 64; ++i) enc[64 * p + i] = e[i];
    }
}

// CTAs of a persistent launch: resident CTAs per SM x SMs, at most one per
// tile; 0 (with the error set) if a query fails.  Residency is computed from
// the kernel's registers and shared memory and the device's limits (the
// occupancy query answers one CTA per SM for the forward kernel, which runs
// six), and capped at `tmem_cap` CTAs (tensor-memory columns per SM).
int persistent_ctas(const void* kernel, int threads, size_t shm, int64_t tiles, int tmem_cap) {
    cudaFuncAttributes fa;
    int dev = 0, regs_sm = 0, smem_sm = 0, smem_res = 0, max_blocks = 0;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_res, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_blocks, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
    if (e != cudaSuccess) {
        set_error("occupancy query failed: %s", cudaGetErrorString(e));
        return 0;
    }
    const int warps = (threads + 31) / 32;
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;  // allocated per warp in units of 256
    const int by_regs = regs_warp > 0 ? regs_sm / (regs_warp * warps) : max_blocks;
    const size_t smem_block = fa.sharedSizeBytes + shm + (size_t)smem_res;
    const int by_smem = smem_block > 0 ? (int)((size_t)smem_sm / smem_block) : max_blocks;
    int per_sm = by_regs < by_smem ? by_regs : by_smem;
    if (per_sm > max_blocks) per_sm = max_blocks;
    if (per_sm > tmem_cap) per_sm = tmem_cap;
    if (per_sm < 1) per_sm = 1;
    return (int)min64((int64_t)per_sm * sm_count(), tiles > 0 ? tiles : 1);
}

}  // namespace

unsigned int mlp_take_status() {
    unsigned int v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_nacc_mlp_status, sizeof(v)) != cudaSuccess) return 0;
    cudaMemcpyToSymbol(g_nacc_mlp_status, &zero, sizeof(zero));
    return v;
}

}  // namespace nacc

using namespace nacc;

extern "C" int nacc_mlp_sync(const float* params, uint16_t* weights, void* stream) {
    clear_error();
    NACC_CHECK_ARG(params && weights, "params / weights is NULL");
    k_mlp_sync<<<33, 256, 0, as_stream(stream)>>>(params, weights);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}

namespace nacc {
namespace {
int launch_forward(int64_t n, const PointSrc& S, const float* params, const uint16_t* weights, float* sigma,
                   cudaStream_t st) {
    const size_t shm = 2 * kWBytes + kTileBytes + 1024;
    const auto kern = S.enc ? k_mlp_forward<true> : k_mlp_forward<false>;
    NACC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    NACC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared));
    const int64_t tiles = (n + kTile - 1) / kTile;
    // at most 8 CTAs of 64 tensor-memory columns share an SM's 512 columns
    const int grid = persistent_ctas((const void*)kern, kThreads, shm, tiles, 8);
    if (grid == 0) return NACC_ERR_CUDA;
    kern<<<grid, kThreads, shm, st>>>(n, S, params, weights, sigma);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}
}  // namespace
}  // namespace nacc

namespace nacc {
namespace {
int forward_rays(int64_t n_rays, int32_t n_bins, const float* rays_o, const float* rays_d, const float* edges,
                 const float* params, const uint16_t* weights, float* sigma, int contract, void* stream) {
    clear_error();
    NACC_CHECK_ARG(n_rays >= 0 && n_rays < (int64_t(1) << 34), "n_rays=%lld out of range", (long long)n_rays);
    NACC_CHECK_ARG(n_bins >= 1 && n_bins <= 4096, "n_bins=%d outside [1, 4096]", n_bins);
    if (n_rays == 0) return NACC_OK;
    NACC_CHECK_ARG(rays_o && rays_d && edges && params && weights && sigma, "a pointer argument is NULL");
    PointSrc S{nullptr, rays_o, rays_d, edges, n_bins, contract, n_rays * n_bins < (int64_t(1) << 32) ? 1 : 0};
    return launch_forward(n_rays * n_bins, S, params, weights, sigma, as_stream(stream));
}
}  // namespace
}  // namespace nacc

extern "C" int nacc_mlp_forward_rays(int64_t n_rays, int32_t n_bins, const float* rays_o, const float* rays_d,
                                     const float* edges, const float* params, const uint16_t* weights,
                                     float* sigma, void* stream) {
    return forward_rays(n_rays, n_bins, rays_o, rays_d, edges, params, weights, sigma, 0, stream);
}

extern "C" int nacc_mlp_forward_rays_contracted(int64_t n_rays, int32_t n_bins, const float* rays_o,
                                                const float* rays_d, const float* edges, const float* params,
                                                const uint16_t* weights, float* sigma, void* stream) {
    return forward_rays(n_rays, n_bins, rays_o, rays_d, edges, params, weights, sigma, 1, stream);
}

extern "C" int nacc_mlp_forward(int64_t n, const float* xyz, const float* params, const uint16_t* weights,
                                float* sigma, void* stream) {
    clear_error();
    NACC_CHECK_ARG(n >= 0 && n < (int64_t(1) << 40), "n=%lld out of range", (long long)n);
    if (n == 0) return NACC_OK;
    NACC_CHECK_ARG(xyz && params && weights && sigma, "a pointer argument is NULL");
    PointSrc S{xyz, nullptr, nullptr, nullptr, 1, 0, 1};
    return launch_forward(n, S, params, weights, sigma, as_stream(stream));
}

namespace nacc {
namespace {
int launch_train(int64_t n, const float* xyz, const uint16_t* enc, const float* target, const float* params,
                 const uint16_t* weights, float* grads, float* loss_sum, cudaStream_t st) {
    NACC_CUDA_TRY(
        cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem));
    const int64_t tiles = (n + kTile - 1) / kTile;
    // one CTA per SM (256 tensor-memory columns each, 138 KiB of shared memory)
    const int grid = (int)min64((int64_t)sm_count(), tiles);
    k_mlp_train<<<grid, kThreads, kTrainSmem, st>>>(n, xyz, enc, target, params, weights, grads, loss_sum,
                                                    (float)(2.0 / (double)n));
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}
}  // namespace
}  // namespace nacc

extern "C" int nacc_mlp_train_grads(int64_t n, const float* xyz, const float* target, const float* params,
                                    const uint16_t* weights, float* grads, float* loss_sum, void* stream) {
    clear_error();
    NACC_CHECK_ARG(n >= 0 && n < (int64_t(1) << 40), "n=%lld out of range", (long long)n);
    if (n == 0) return NACC_OK;
    NACC_CHECK_ARG(xyz && target && params && weights && grads && loss_sum, "a pointer argument is NULL");
    return launch_train(n, xyz, nullptr, target, params, weights, grads, loss_sum, as_stream(stream));
}

extern "C" int nacc_mlp_forward_encoded(int64_t n, const uint16_t* enc, const float* params,
                                        const uint16_t* weights, float* sigma, void* stream) {
    clear_error();
    NACC_CHECK_ARG(n >= 0 && n < (int64_t(1) << 40), "n=%lld out of range", (long long)n);
    if (n == 0) return NACC_OK;
    NACC_CHECK_ARG(enc && params && weights && sigma, "a pointer argument is NULL");
    NACC_CHECK_ARG((reinterpret_cast<uintptr_t>(enc) & 15) == 0, "enc must be 16-byte aligned");
    PointSrc S{nullptr, nullptr, nullptr, nullptr, 1, 0, 1, enc};
    return launch_forward(n, S, params, weights, sigma, as_stream(stream));
}

extern "C" int nacc_mlp_train_grads_encoded(int64_t n, const uint16_t* enc, const float* target,
                                            const float* params, const uint16_t* weights, float* grads,
                                            float* loss_sum, void* stream) {
    clear_error();
    NACC_CHECK_ARG(n >= 0 && n < (int64_t(1) << 40), "n=%lld out of range", (long long)n);
    if (n == 0) return NACC_OK;
    NACC_CHECK_ARG(enc && target && params && weights && grads && loss_sum, "a pointer argument is NULL");
    NACC_CHECK_ARG((reinterpret_cast<uintptr_t>(enc) & 15) == 0, "enc must be 16-byte aligned");
    return launch_train(n, nullptr, enc, target, params, weights, grads, loss_sum, as_stream(stream));
}

extern "C" int nacc_mlp_adam(float* params, float* grads, float* m, float* v, int64_t step, float lr, float beta1,
                             float beta2, float eps, uint16_t* weights, void* stream) {
    clear_error();
    NACC_CHECK_ARG(params && grads && m && v && weights, "a pointer argument is NULL");
    NACC_CHECK_ARG(step >= 1, "step=%lld must be >= 1", (long long)step);
    NACC_CHECK_ARG(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f, "betas outside [0, 1)");
    const float bc1 = (float)(1.0 - std::pow((double)beta1, (double)step));
    const float bc2 = (float)(1.0 - std::pow((double)beta2, (double)step));
    k_mlp_adam<<<33, 256, 0, as_stream(stream)>>>(params, grads, m, v, lr, beta1, beta2, eps, bc1, bc2, weights);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}

extern "C" int nacc_mlp_encode(int64_t n, const float* xyz, float* enc, void* stream) {
    clear_error();
    NACC_CHECK_ARG(n >= 0 && n < (int64_t(1) << 40), "n=%lld out of range", (long long)n);
    if (n == 0) return NACC_OK;
    NACC_CHECK_ARG(xyz && enc, "xyz / enc is NULL");
    const int blocks = (int)min64((n + 255) / 256, (int64_t)sm_count() * 8);
    k_mlp_encode<<<blocks, 256, 0, as_stream(stream)>>>(n, xyz, enc);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}
