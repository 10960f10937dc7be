// The warm-start U-Net on the GPU: forward, backward and Adam, with every
// 3x3 convolution an implicit GEMM on the tensor cores (BF16 operands, FP32
// accumulation) with tcgen05 and the accumulator in tensor memory: forward
// and data gradient with K-major operands, the weight gradient with MN-major
// ones read straight from the NHWC tensors.  The remaining layers (pooling,
// upsampling with concatenation, the 1x1 head, the loss, Adam) are small
// kernels of their own.
//
// Layout: activations NHWC in BF16 (channels innermost, every channel count
// a multiple of 8, so that 8 channels are one 16-byte load); conv weights
// [Cout][tap][Cin] (tap = 3 ky + kx) in BF16, with a transposed copy
// [Cin][tap][Cout] for the backward pass over the data; FP32 master weights,
// gradients and Adam moments in the same layout.
//
// Convolutions as GEMMs (P = B H W pixels, s(tap) = (ky - 1, kx - 1)):
//   forward      out[p][co]  = sum_{tap,ci} x[p + s][ci] w[co][tap][ci]        M=P  N=Cout K=9 Cin
//   data grad    dx[p][ci]   = sum_{tap,co} dz[p - s][co] w[co][tap][ci]       M=P  N=Cin  K=9 Cout
//   weight grad  dw[co][tap][ci] = sum_p dz[p][co] x[p + s][ci]                M=Cout N=9 Cin K=P
// (zero outside the image).  The weight gradient splits K over blocks and
// adds FP32 partial sums atomically.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "lbm_nn.h"

namespace nn {

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------ GEMM core

constexpr int BM = 64, BN = 64, BK = 32, LDS = BK + 8;  // smem rows padded by 16 bytes
constexpr int GEMM_THREADS = 128;                       // 2 x 2 warps of 32 x 32

struct alignas(16) Tiles {
    bf16 a[BM][LDS];
    bf16 b[BN][LDS];
};

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__device__ __forceinline__ void ldsm_x2(uint32_t (&r)[2], const void *p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r[0]), "=r"(r[1])
                 : "r"(a));
}

// C[M][N] = sum_k A[m][k] B[n][k] over this block's K range; the operation
// Op gathers the tiles (load_a, load_b) and consumes the result (store).
template <class Op>
__global__ void __launch_bounds__(GEMM_THREADS) k_gemm(const Op op) {
    __shared__ Tiles t;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    int kb = 0, ke = op.K;
    if (gridDim.z > 1) {
        kb = blockIdx.z * op.kchunk;
        ke = min(op.K, kb + op.kchunk);
    }
    float c[2][4][4] = {};
    for (int k0 = kb; k0 < ke; k0 += BK) {
        op.load_a(t.a, m0, k0, ke, tid);
        op.load_b(t.b, n0, k0, ke, tid);
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; mi++)
                ldsm_x4(af[mi], &t.a[wm * 32 + mi * 16 + (lane & 15)][ks + (lane >> 4) * 8]);
#pragma unroll
            for (int ni = 0; ni < 4; ni++)
                ldsm_x2(bfr[ni], &t.b[wn * 32 + ni * 8 + (lane & 7)][ks + ((lane >> 3) & 1) * 8]);
#pragma unroll
            for (int mi = 0; mi < 2; mi++)
#pragma unroll
                for (int ni = 0; ni < 4; ni++) mma_bf16(c[mi][ni], af[mi], bfr[ni]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int mi = 0; mi < 2; mi++)
#pragma unroll
        for (int ni = 0; ni < 4; ni++) {
            const int r = m0 + wm * 32 + mi * 16 + (lane >> 2);
            const int col = n0 + wn * 32 + ni * 8 + (lane & 3) * 2;
            op.store(r, col, c[mi][ni][0], c[mi][ni][1]);
            op.store(r + 8, col, c[mi][ni][2], c[mi][ni][3]);
        }
}

// Geometry of an NHWC image batch.
struct Img {
    int B, H, W;
    __device__ __forceinline__ bool shift(int p, int dy, int dx, int &q) const {
        const int hw = H * W;
        const int n = p / hw, r = p - n * hw, y = r / W, x = r - y * W;
        const int ys = y + dy, xs = x + dx;
        if (ys < 0 || ys >= H || xs < 0 || xs >= W) return false;
        q = (n * H + ys) * W + xs;
        return true;
    }
};

// Forward convolution (sign = +1) or the gradient with respect to its input
// (sign = -1, w the transposed weights): out[p][n] = act(bias + sum over taps
// and source channels of src[p + sign s(tap)][c] w[n][tap][c]), times
// (mask > 0) when a mask is given.
struct ConvOp {
    const bf16 *src;   // [P][Cs]
    const bf16 *w;     // [N][taps][Cs]
    const float *bias; // [N] or null
    const bf16 *mask;  // [P][N] or null
    bf16 *out;         // [P][N]
    Img img;
    int Cs, taps, sign, relu;
    int M, N, K, kchunk;

    // 8 consecutive K elements of row p of A (source channels of one tap)
    __device__ __forceinline__ uint4 gather_a(int p, int k, int ke) const {
        uint4 v = make_uint4(0, 0, 0, 0);
        if (p < M && k < ke) {
            const int tap = k / Cs, c = k - tap * Cs;
            int qp = p;
            bool ok = true;
            if (taps == 9) ok = img.shift(p, sign * (tap / 3 - 1), sign * (tap % 3 - 1), qp);
            if (ok) v = *reinterpret_cast<const uint4 *>(src + (size_t)qp * Cs + c);
        }
        return v;
    }
    // address of the 8 K elements of row p of A, or null where they are zero
    __device__ __forceinline__ const bf16 *addr_a(int p, int k, int ke) const {
        if (p >= M || k >= ke) return nullptr;
        const int tap = k / Cs, c = k - tap * Cs;
        int qp = p;
        if (taps == 9 && !img.shift(p, sign * (tap / 3 - 1), sign * (tap % 3 - 1), qp)) return nullptr;
        return src + (size_t)qp * Cs + c;
    }
    __device__ __forceinline__ const bf16 *addr_b(int n, int k, int ke) const {
        return (n < N && k < ke) ? w + (size_t)n * K + k : nullptr;
    }
    // 8 consecutive K elements of row n of B (the weights of one output)
    __device__ __forceinline__ uint4 gather_b(int n, int k, int ke) const {
        uint4 v = make_uint4(0, 0, 0, 0);
        if (n < N && k < ke) v = *reinterpret_cast<const uint4 *>(w + (size_t)n * K + k);
        return v;
    }
    __device__ __forceinline__ void load_a(bf16 (&a)[BM][LDS], int m0, int k0, int ke, int tid) const {
#pragma unroll
        for (int i = 0; i < 2; i++) {
            const int q = tid + i * GEMM_THREADS, r = q >> 2, cc = q & 3;
            *reinterpret_cast<uint4 *>(&a[r][cc * 8]) = gather_a(m0 + r, k0 + cc * 8, ke);
        }
    }
    __device__ __forceinline__ void load_b(bf16 (&b)[BN][LDS], int n0, int k0, int ke, int tid) const {
#pragma unroll
        for (int i = 0; i < 2; i++) {
            const int q = tid + i * GEMM_THREADS, r = q >> 2, cc = q & 3;
            *reinterpret_cast<uint4 *>(&b[r][cc * 8]) = gather_b(n0 + r, k0 + cc * 8, ke);
        }
    }
    // epilogue of 16 consecutive outputs (n multiple of 8, N a multiple of 8)
    __device__ __forceinline__ void store16(int m, int n, const float *v) const {
        if (m >= M) return;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int nh = n + 8 * h;
            if (nh >= N) return;
            float o[8];
#pragma unroll
            for (int j = 0; j < 8; j++) {
                o[j] = v[8 * h + j];
                if (bias) o[j] += bias[nh + j];
                if (relu) o[j] = fmaxf(o[j], 0.f);
            }
            const size_t off = (size_t)m * N + nh;
            if (mask) {
                const uint4 mk = *reinterpret_cast<const uint4 *>(mask + off);
                const bf16 *me = reinterpret_cast<const bf16 *>(&mk);
#pragma unroll
                for (int j = 0; j < 8; j++)
                    if (!(__bfloat162float(me[j]) > 0.f)) o[j] = 0.f;
            }
            uint4 pk;
            __nv_bfloat162 *pp = reinterpret_cast<__nv_bfloat162 *>(&pk);
#pragma unroll
            for (int j = 0; j < 4; j++) pp[j] = __floats2bfloat162_rn(o[2 * j], o[2 * j + 1]);
            *reinterpret_cast<uint4 *>(out + off) = pk;
        }
    }
    __device__ __forceinline__ void store(int m, int n, float v0, float v1) const {
        if (m >= M || n >= N) return;
        if (bias) {
            v0 += bias[n];
            v1 += bias[n + 1];
        }
        if (relu) {
            v0 = fmaxf(v0, 0.f);
            v1 = fmaxf(v1, 0.f);
        }
        const size_t o = (size_t)m * N + n;
        if (mask) {
            const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162 *>(mask + o);
            if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
            if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
        }
        *reinterpret_cast<__nv_bfloat162 *>(out + o) = __floats2bfloat162_rn(v0, v1);
    }
};

// Weight gradient: dw[co][tap][c] += sum_p dz[p][co] x[p + s(tap)][c] over
// this block's pixel range (K = pixels).
struct WgradOp {
    const bf16 *dz;  // [P][Co]
    const bf16 *x;   // [P][Ci]
    float *dw;       // [Co][taps][Ci]
    Img img;
    int Co, Ci, taps;
    int M, N, K, kchunk;  // M = Co, N = taps Ci, K = P

    __device__ __forceinline__ void load_a(bf16 (&a)[BM][LDS], int m0, int k0, int ke, int tid) const {
        // 32 pixels x 64 output channels: chunk (pixel, 8 channels), transposed into a[co][pixel]
#pragma unroll
        for (int i = 0; i < 2; i++) {
            const int q = tid + i * GEMM_THREADS, pl = q >> 3, cc = q & 7;
            const int p = k0 + pl, co = m0 + cc * 8;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (p < ke && co < M) v = *reinterpret_cast<const uint4 *>(dz + (size_t)p * Co + co);
            const bf16 *e = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
            for (int j = 0; j < 8; j++) a[cc * 8 + j][pl] = e[j];
        }
    }
    __device__ __forceinline__ void load_b(bf16 (&b)[BN][LDS], int n0, int k0, int ke, int tid) const {
#pragma unroll
        for (int i = 0; i < 2; i++) {
            const int q = tid + i * GEMM_THREADS, pl = q >> 3, cc = q & 7;
            const int p = k0 + pl, n = n0 + cc * 8;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (p < ke && n < N) {
                const int tap = n / Ci, c = n - tap * Ci;
                int qp = p;
                bool ok = true;
                if (taps == 9) ok = img.shift(p, tap / 3 - 1, tap % 3 - 1, qp);
                if (ok) v = *reinterpret_cast<const uint4 *>(x + (size_t)qp * Ci + c);
            }
            const bf16 *e = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
            for (int j = 0; j < 8; j++) b[cc * 8 + j][pl] = e[j];
        }
    }
    __device__ __forceinline__ void store(int m, int n, float v0, float v1) const {
        if (m >= M || n >= N) return;
        atomicAdd(dw + (size_t)m * N + n, v0);
        atomicAdd(dw + (size_t)m * N + n + 1, v1);
    }
};

// ------------------------------------------------ tcgen05 convolution
//
// The forward and data-gradient convolutions (ConvOp) on the 5th-generation
// tensor cores: a CTA of 128 threads owns a 128 x BN output tile whose FP32
// accumulator lives in tensor memory (BN columns allocated per CTA).  Each K
// block of 64 is gathered into shared memory with cp.async (16 bytes per
// copy, zero-filled outside the image) in the K-major no-swizzle layout of
// 8 x 16-byte core matrices (core matrix (row group g, K group j) at
// g * 1024 + j * 128 bytes); one thread then issues four
// tcgen05.mma.kind::f16 (M = 128, N = BN, K = 16; BF16 in, FP32 accumulate)
// and commits them to the stage's mbarrier.  TC_STAGES stages: the copies of
// the next blocks are in flight while the tensor cores work.  Every mbarrier
// wait is bounded (by the network's wait limit, a number of polls); a wait
// that runs out stops the pipeline, the CTA waits (bounded by TC_SPIN) for the
// MMAs it has issued, frees its tensor memory, sets *err and stores nothing.
constexpr int TC_M = 128, TC_K = 64, TC_THREADS = 256, TC_STAGES = 3;
constexpr int TC_TABLE_MAX = 8192;  // bytes of the A operand's K table (K up to 8192)
constexpr long long TC_SPIN = 1 << 24;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: K-major, no swizzle, 128 B between K
// groups (leading), 1024 B between 8-row groups (stride)
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity, long long limit) {
    uint32_t done = 0;
    for (long long it = 0; it < limit && !done; it++)
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
    return done != 0;
}

// 16-byte global -> shared copy; a null source fills zeros
__device__ __forceinline__ void cp16(uint32_t dst, const void *src, const void *dummy) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst),
                 "l"(src ? src : dummy), "r"(src ? 16 : 0)
                 : "memory");
}

// The MMA pipeline of the tcgen05 kernels: TC_STAGES shared-memory stages
// filled with cp.async by every thread (stage(i, addr) copies K block i; it is
// called for i = 0, 1, 2, ... in order), one thread issuing a block's four
// K = 16 MMAs (mma(addr, accumulate)) and committing them to the stage's
// mbarrier, which is waited for (at most `limit` polls) before the stage is
// refilled.  The block of iteration j completes phase j / TC_STAGES of barrier
// j % TC_STAGES, and every barrier has at most one phase outstanding when it
// is waited for.  A wait that gives up in any thread ends the pipeline before
// the next MMA (no stage is refilled while the tensor cores may read it);
// the issuing thread then commits once more to the drain barrier
// mbar[TC_STAGES], which completes when every MMA it issued has, and the CTA
// waits for that (at most TC_SPIN polls) before its tensor memory is read or
// freed.  Returns false, in every thread, when a wait gave up.
template <int STAGE, class StageFn, class MmaFn>
__device__ __forceinline__ bool tc_pipeline(int nk, uint32_t base, uint64_t *mbar, int tid,
                                            long long limit, StageFn &&stage, MmaFn &&mma) {
    bool ok = true;
    int issued = 0;  // K blocks whose MMAs were issued (the same in every thread)
#pragma unroll
    for (int st = 0; st < TC_STAGES - 1; st++) {
        if (st < nk) stage(st, base + st * STAGE);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    for (int kt = 0; kt < nk; kt++) {
        const int s = kt % TC_STAGES;
        asm volatile("cp.async.wait_group %0;\n" ::"n"(TC_STAGES - 2) : "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        if (__syncthreads_or(!ok)) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            mma(base + s * STAGE, kt > 0);
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(&mbar[s])));
        }
        issued = kt + 1;
        // refill the stage of block kt - 1 once its MMAs are done
        const int nxt = kt + TC_STAGES - 1;
        if (nxt < nk) {
            if (kt > 0)
                ok &= tc_wait(smem_u32(&mbar[(kt - 1) % TC_STAGES]), ((kt - 1) / TC_STAGES) & 1,
                              limit);
            if (ok) stage(nxt, base + (nxt % TC_STAGES) * STAGE);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    // blocks max(nk - TC_STAGES, 0) .. nk - 1 have not been waited for
    if (issued == nk)
        for (int j = nk > TC_STAGES ? nk - TC_STAGES : 0; j < nk; j++)
            ok &= tc_wait(smem_u32(&mbar[j % TC_STAGES]), (j / TC_STAGES) & 1, limit);
    ok = __syncthreads_and(ok);
    if (!ok) {
        if (tid == 0)
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    smem_u32(&mbar[TC_STAGES])));
        tc_wait(smem_u32(&mbar[TC_STAGES]), 0, TC_SPIN);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    return ok;
}

__device__ __forceinline__ void tc_alloc(uint32_t *slot, uint64_t *mbar, int ncols, int warp, int tid) {
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(slot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int s = 0; s <= TC_STAGES; s++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[s])));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
}

__device__ __forceinline__ void tc_free(uint32_t tmem, int ncols, int warp) {
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols));
}

// 16 consecutive FP32 accumulator columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tc_ld16(uint32_t addr, float (&f)[16]) {
    uint32_t v[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; j++) f[j] = __uint_as_float(v[j]);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                       uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// Shared-memory table of the K axis of a convolution's A operand, one entry
// per 8 consecutive K elements: the element offset of the 8 source channels
// from the row's own pixel, and the index 3 dy + dx + 4 of the displacement
// (31 beyond K, which no row's bounds mask has).
__device__ __forceinline__ void conv_table(const ConvOp &op, int2 *tab, int nent, int tid) {
    for (int e = tid; e < nent; e += TC_THREADS) {
        int2 v = make_int2(0, 31);
        if (8 * e < op.K) {
            const int k = 8 * e, tap = k / op.Cs, c = k - tap * op.Cs;
            const int dy = op.taps == 9 ? op.sign * (tap / 3 - 1) : 0;
            const int dx = op.taps == 9 ? op.sign * (tap % 3 - 1) : 0;
            v = make_int2((dy * op.img.W + dx) * op.Cs + c, 3 * dy + dx + 4);
        }
        tab[e] = v;
    }
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS) k_conv_tc(const ConvOp op, long long limit, int *err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t mbar[TC_STAGES + 1];  // the stages' and the drain barrier
    constexpr int STAGE = TC_M * TC_K * 2 + BN * TC_K * 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_M, n0 = blockIdx.y * BN;
    const uint32_t base = smem_u32(smem);
    const int nk = (op.K + TC_K - 1) / TC_K, nkk = op.K >> 3;
    int2 *tab = reinterpret_cast<int2 *>(smem + TC_STAGES * STAGE);
    conv_table(op, tab, nk * (TC_K / 8), tid);
    // Copies: lanes l and l + 16 of a warp take 8-channel chunks 2j and 2j + 1
    // of one row, so a warp reads 16 rows x 32 contiguous bytes (whole
    // sectors) and each 8-lane phase writes 8 rows of one core matrix.
    // This thread's A row (a pixel) and its 3x3 neighbours inside the image:
    const int r = 16 * warp + (lane & 15), p = m0 + r;
    uint32_t inb = 0;
    const bf16 *arow = op.src;
    if (p < op.M) {
        const int hw = op.img.H * op.img.W, q = p % hw, y = q / op.img.W, x = q - y * op.img.W;
#pragma unroll
        for (int b = 0; b < 9; b++) {
            const int ys = y + b / 3 - 1, xs = x + b % 3 - 1;
            if (ys >= 0 && ys < op.img.H && xs >= 0 && xs < op.img.W) inb |= 1u << b;
        }
        arow = op.src + (size_t)p * op.Cs;
    }
    // this thread's B row (an output channel) and first chunk pair
    const int rb = 16 * (warp % (BN / 16)) + (lane & 15), nb = n0 + rb, kpb = warp / (BN / 16);
    const bf16 *brow = op.w + (size_t)(nb < op.N ? nb : 0) * op.K;
    tc_alloc(&tmem_base, mbar, BN, warp, tid);  // its barrier also publishes the table
    const uint32_t tmem = tmem_base;
    // kind::f16: D FP32, A and B BF16, both K-major, N = BN, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(TC_M >> 4) << 24);
    auto stage = [&](int kt, uint32_t sa) {
        const uint32_t sb = sa + TC_M * TC_K * 2;
        const int kk0 = kt * (TC_K / 8);
#pragma unroll
        for (int i = 0; i < TC_M * 8 / TC_THREADS; i++) {
            const int kg = 2 * i + (lane >> 4);
            const int2 e = tab[kk0 + kg];
            cp16(sa + (r >> 3) * 1024 + kg * 128 + (r & 7) * 16,
                 ((inb >> e.y) & 1u) ? arow + e.x : nullptr, op.src);
        }
#pragma unroll
        for (int i = 0; i < BN * 8 / TC_THREADS; i++) {
            const int kg = 2 * (kpb + (TC_M / BN) * i) + (lane >> 4), kk = kk0 + kg;
            cp16(sb + (rb >> 3) * 1024 + kg * 128 + (rb & 7) * 16,
                 (nb < op.N && kk < nkk) ? brow + 8 * kk : nullptr, op.w);
        }
    };
    auto mma = [&](uint32_t sa, bool accumulate) {
        const uint32_t sb = sa + TC_M * TC_K * 2;
#pragma unroll
        for (int ks = 0; ks < TC_K / 16; ks++)
            tc_mma(tmem, tc_desc(sa + ks * 256), tc_desc(sb + ks * 256), idesc,
                   (accumulate || ks > 0) ? 1u : 0u);
    };
    const bool ok = tc_pipeline<STAGE>(nk, base, mbar, tid, limit, stage, mma);
    if (!ok) atomicOr(err, 1);
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, columns of half w / 4
    const int row = m0 + (warp & 3) * 32 + lane, cb = (warp >> 2) * (BN / 2);
#pragma unroll
    for (int c0 = 0; c0 < BN / 2; c0 += 16) {
        float f[16];
        tc_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + cb + c0, f);
        if (ok && n0 + cb + c0 < op.N) op.store16(row, n0 + cb + c0, f);
    }
    tc_free(tmem, BN, warp);
}

// Weight gradient on tcgen05: dw[co][tap][ci] += sum_p x[p + s(tap)][ci] dz[p][co],
// i.e. D[m][n] with m = (tap, ci) (M = taps Cin), n = co, K = pixels.  Both
// operands are MN-major in shared memory (8 consecutive channels of one
// pixel form a 16-byte core-matrix row), so they are copied straight from the
// NHWC tensors: core matrix (MN group g, K group j) at j * LBO + g * 128
// bytes, LBO = (rows / 8) * 128.  The pixel range of a block is one split of
// K (gridDim.z); results are added to dw with FP32 atomics.
struct WgradTc {
    const bf16 *dz;  // [P][Co]
    const bf16 *x;   // [P][Ci]
    float *dw;       // [Co][taps][Ci]
    Img img;
    int Co, Ci, taps, M, N, K, kchunk;  // M = taps Ci, N = Co, K = P
};

template <int BN>
__global__ void __launch_bounds__(TC_THREADS) k_wgrad_tc(const WgradTc op, long long limit, int *err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t mbar[TC_STAGES + 1];  // the stages' and the drain barrier
    constexpr int STAGE = TC_M * TC_K * 2 + BN * TC_K * 2;
    constexpr int AG = TC_M * TC_K / 8 / TC_THREADS, BG = BN * TC_K / 8 / TC_THREADS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_M, n0 = blockIdx.y * BN;
    const int kb = blockIdx.z * op.kchunk, ke = min(op.K, kb + op.kchunk);
    const int nk = ke > kb ? (ke - kb + TC_K - 1) / TC_K : 0;
    const uint32_t base = smem_u32(smem);
    // This thread copies pixel pl of every K block, channel groups
    // g = 2 (w / 4 + 2 i) + l / 16 (warp w, lane l): lanes l and l + 16 take
    // adjacent groups of one pixel (32 contiguous bytes), and each 8-lane
    // phase writes 8 pixels of one core matrix.  The (tap, channel) of each A
    // group is fixed: its offset from the pixel and displacement (dy, dx).
    const int pl = 16 * (warp & 3) + (lane & 15), g0 = 2 * (warp >> 2) + (lane >> 4);
    int aoff[AG], ady[AG], adx[AG];
#pragma unroll
    for (int i = 0; i < AG; i++) {
        const int m = m0 + 8 * (g0 + 4 * i);
        aoff[i] = 0;
        ady[i] = 1 << 20;  // never inside the image
        adx[i] = 0;
        if (m < op.M) {
            const int tap = m / op.Ci, c = m - tap * op.Ci;
            ady[i] = op.taps == 9 ? tap / 3 - 1 : 0;
            adx[i] = op.taps == 9 ? tap % 3 - 1 : 0;
            aoff[i] = (ady[i] * op.img.W + adx[i]) * op.Ci + c;
        }
    }
    // coordinates of this thread's pixel, advanced by TC_K per block
    int p = kb + pl, xx = p % op.img.W, yy = (p / op.img.W) % op.img.H;
    tc_alloc(&tmem_base, mbar, BN < 32 ? 32 : BN, warp, tid);
    const uint32_t tmem = tmem_base;
    // kind::f16: D FP32, A and B BF16, both MN-major, N = BN, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                           ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
    auto stage = [&](int, uint32_t sa) {
        const uint32_t sb = sa + TC_M * TC_K * 2;
        const bool pv = p < ke;
#pragma unroll
        for (int i = 0; i < AG; i++) {
            const int g = g0 + 4 * i;
            const bool in = pv && (unsigned)(yy + ady[i]) < (unsigned)op.img.H &&
                            (unsigned)(xx + adx[i]) < (unsigned)op.img.W;
            cp16(sa + (pl >> 3) * (TC_M / 8 * 128) + g * 128 + (pl & 7) * 16,
                 in ? op.x + (size_t)p * op.Ci + aoff[i] : nullptr, op.x);
        }
#pragma unroll
        for (int i = 0; i < BG; i++) {
            const int g = g0 + 4 * i, n = n0 + 8 * g;
            cp16(sb + (pl >> 3) * (BN / 8 * 128) + g * 128 + (pl & 7) * 16,
                 (pv && n < op.N) ? op.dz + (size_t)p * op.Co + n : nullptr, op.dz);
        }
        p += TC_K;
        xx += TC_K;
        while (xx >= op.img.W) {
            xx -= op.img.W;
            if (++yy == op.img.H) yy = 0;
        }
    };
    auto mma = [&](uint32_t sa, bool accumulate) {
        const uint32_t sb = sa + TC_M * TC_K * 2;
#pragma unroll
        for (int ks = 0; ks < TC_K / 16; ks++) {
            // two K groups per MMA; leading offset = K-group stride, stride offset = 128
            uint64_t ad = (uint64_t)(((sa + ks * 2 * (TC_M / 8 * 128)) >> 4) & 0x3FFF);
            ad |= (uint64_t)((TC_M / 8 * 128) >> 4) << 16;
            ad |= (uint64_t)(128 >> 4) << 32;
            ad |= (uint64_t)1 << 46;
            uint64_t bd = (uint64_t)(((sb + ks * 2 * (BN / 8 * 128)) >> 4) & 0x3FFF);
            bd |= (uint64_t)((BN / 8 * 128) >> 4) << 16;
            bd |= (uint64_t)(128 >> 4) << 32;
            bd |= (uint64_t)1 << 46;
            tc_mma(tmem, ad, bd, idesc, (accumulate || ks > 0) ? 1u : 0u);
        }
    };
    const bool ok = tc_pipeline<STAGE>(nk, base, mbar, tid, limit, stage, mma);
    if (!ok) atomicOr(err, 1);
    const int m = m0 + (warp & 3) * 32 + lane, cb = (warp >> 2) * (BN / 2);
#pragma unroll
    for (int c0 = 0; c0 < BN / 2; c0 += 16) {
        float f[16];
        tc_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + cb + c0, f);
        if (ok && m < op.M && nk > 0) {
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int n = n0 + cb + c0 + j;
                if (n < op.N) atomicAdd(op.dw + (size_t)n * op.M + m, f[j]);
            }
        }
    }
    tc_free(tmem, BN < 32 ? 32 : BN, warp);
}

// ------------------------------------------------------ other layers

constexpr int EW = 256;  // threads of the elementwise kernels

inline unsigned blocks(long long n) { return (unsigned)((n + EW - 1) / EW); }

// NCHW float input [B][8][H][W] -> NHWC BF16 [P][8]
__global__ void k_pack_input(const float *in, bf16 *x, int B, int HW) {
    const long long i = (long long)blockIdx.x * EW + threadIdx.x;
    if (i >= (long long)B * HW * 8) return;
    const int c = (int)(i & 7);
    const long long p = i >> 3, n = p / HW, r = p - n * HW;
    x[i] = __float2bfloat16(in[(n * 8 + c) * HW + r]);
}

// The NHWC layers below work on groups of 8 channels (one 16-byte word);
// every channel count is a multiple of 8.
__device__ __forceinline__ void unpack8(const uint4 &v, float (&f)[8]) {
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const float2 t = __bfloat1622float2(h[j]);
        f[2 * j] = t.x;
        f[2 * j + 1] = t.y;
    }
}
__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
    uint4 v;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&v);
#pragma unroll
    for (int j = 0; j < 4; j++) h[j] = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
    return v;
}

// 2x2 average pooling of NHWC [B][H][W][C] into [B][H/2][W/2][C]
__global__ void k_pool(const bf16 *in, bf16 *out, int B, int H, int W, int C) {
    const int G = C / 8, Ho = H / 2, Wo = W / 2;
    const long long i = (long long)blockIdx.x * EW + threadIdx.x;
    if (i >= (long long)B * Ho * Wo * G) return;
    const int g = (int)(i % G);
    const long long p = i / G;
    const int x = (int)(p % Wo), y = (int)((p / Wo) % Ho);
    const long long n = p / ((long long)Wo * Ho);
    const long long b0 = ((n * H + 2 * y) * W + 2 * x) * C + 8 * g;
    float a[8], t[8];
    unpack8(*reinterpret_cast<const uint4 *>(in + b0), a);
    const long long offs[3] = {C, (long long)W * C, (long long)W * C + C};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        unpack8(*reinterpret_cast<const uint4 *>(in + b0 + offs[k]), t);
#pragma unroll
        for (int j = 0; j < 8; j++) a[j] += t[j];
    }
#pragma unroll
    for (int j = 0; j < 8; j++) a[j] *= 0.25f;
    *reinterpret_cast<uint4 *>(out + p * C + 8 * g) = pack8(a);
}

// de[p][c] = (e[p][c] > 0) * dpool[p/2][c] / 4 + dskip[p][c] (dskip: a
// channel slice of stride Cs at offset off, already masked)
__global__ void k_pool_back(const bf16 *dpool, const bf16 *e, const bf16 *dskip, int Cs, int off,
                            bf16 *de, int B, int H, int W, int C) {
    const int G = C / 8;
    const long long i = (long long)blockIdx.x * EW + threadIdx.x;
    if (i >= (long long)B * H * W * G) return;
    const int g = (int)(i % G);
    const long long p = i / G;
    const int x = (int)(p % W), y = (int)((p / W) % H);
    const long long n = p / ((long long)W * H);
    const long long q = (n * (H / 2) + y / 2) * (W / 2) + x / 2;
    float dp[8], ev[8], ds[8] = {0, 0, 0, 0, 0, 0, 0, 0}, o[8];
    unpack8(*reinterpret_cast<const uint4 *>(dpool + q * C + 8 * g), dp);
    unpack8(*reinterpret_cast<const uint4 *>(e + p * C + 8 * g), ev);
    if (dskip) unpack8(*reinterpret_cast<const uint4 *>(dskip + p * Cs + off + 8 * g), ds);
#pragma unroll
    for (int j = 0; j < 8; j++) o[j] = (ev[j] > 0.f ? 0.25f * dp[j] : 0.f) + ds[j];
    *reinterpret_cast<uint4 *>(de + p * C + 8 * g) = pack8(o);
}

// cat[p] = [up(d)[p] (Cu channels), e[p] (Ce channels)]
__global__ void k_upcat(const bf16 *d, const bf16 *e, bf16 *cat, int B, int H, int W, int Cu,
                        int Ce) {
    const int Gc = (Cu + Ce) / 8, Gu = Cu / 8;
    const long long i = (long long)blockIdx.x * EW + threadIdx.x;
    if (i >= (long long)B * H * W * Gc) return;
    const int g = (int)(i % Gc);
    const long long p = i / Gc;
    uint4 v;
    if (g < Gu) {
        const int x = (int)(p % W), y = (int)((p / W) % H);
        const long long n = p / ((long long)W * H);
        const long long q = (n * (H / 2) + y / 2) * (W / 2) + x / 2;
        v = *reinterpret_cast<const uint4 *>(d + q * Cu + 8 * g);
    } else {
        v = *reinterpret_cast<const uint4 *>(e + p * Ce + 8 * (g - Gu));
    }
    *reinterpret_cast<uint4 *>(cat + p * (Cu + Ce) + 8 * g) = v;
}

// dd[q][c] = sum over the 2x2 children p of q of dcat[p][c], c < Cu
__global__ void k_up_back(const bf16 *dcat, int Cc, bf16 *dd, int B, int Hc, int Wc, int Cu) {
    const int G = Cu / 8;
    const long long i = (long long)blockIdx.x * EW + threadIdx.x;
    if (i >= (long long)B * Hc * Wc * G) return;
    const int g = (int)(i % G);
    const long long q = i / G;
    const int x = (int)(q % Wc), y = (int)((q / Wc) % Hc);
    const long long n = q / ((long long)Wc * Hc);
    const int H = 2 * Hc, W = 2 * Wc;
    const long long p0 = (n * H + 2 * y) * W + 2 * x;
    const long long ps[4] = {p0, p0 + 1, p0 + W, p0 + W + 1};
    float a[8] = {0, 0, 0, 0, 0, 0, 0, 0}, t[8];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        unpack8(*reinterpret_cast<const uint4 *>(dcat + ps[k] * Cc + 8 * g), t);
#pragma unroll
        for (int j = 0; j < 8; j++) a[j] += t[j];
    }
    *reinterpret_cast<uint4 *>(dd + q * Cu + 8 * g) = pack8(a);
}

// 1x1 head: out[n][o][y][x] = b[o] + sum_c w[o][c] d[p][c] (FP32), NCHW output
__global__ void k_head(const bf16 *d, const float *w, const float *b, float *out, int B, int HW,
                       int C) {
    const long long p = (long long)blockIdx.x * EW + threadIdx.x;
    if (p >= (long long)B * HW) return;
    float acc[3] = {b[0], b[1], b[2]};
    for (int c = 0; c < C; c += 8) {
        const uint4 v = *reinterpret_cast<const uint4 *>(d + p * C + c);
        const bf16 *e = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const float x = __bfloat162float(e[j]);
#pragma unroll
            for (int o = 0; o < 3; o++) acc[o] += w[o * C + c + j] * x;
        }
    }
    const long long n = p / HW, r = p - n * HW;
#pragma unroll
    for (int o = 0; o < 3; o++) out[(n * 3 + o) * HW + r] = acc[o];
}

// fluid-node count (for the loss normalisation)
__global__ void k_count(const float *fluid, long long n, float *cnt) {
    __shared__ float s[EW];
    float a = 0.f;
    for (long long i = (long long)blockIdx.x * EW + threadIdx.x; i < n; i += (long long)gridDim.x * EW)
        a += fluid[i];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int o = EW / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(cnt, s[0]);
}

// loss = sum (out - t)^2 m / (3 count); dout = 2 (out - t) m / (3 count)
__global__ void k_loss(const float *out, const float *tgt, const float *fluid, const float *cnt,
                       float *dout, double *loss, int B, int HW) {
    __shared__ float s[EW];
    const long long n3 = (long long)B * 3 * HW;
    const float inv = 1.f / (3.f * fmaxf(*cnt, 1.f));
    float a = 0.f;
    for (long long i = (long long)blockIdx.x * EW + threadIdx.x; i < n3; i += (long long)gridDim.x * EW) {
        const long long n = i / (3 * HW), r = i % HW;
        const float m = fluid[n * HW + r];
        const float d = (out[i] - tgt[i]) * m;
        a += d * d;
        dout[i] = 2.f * d * inv;
    }
    s[threadIdx.x] = a;
    __syncthreads();
    for (int o = EW / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, (double)(s[0] * inv));
}

// head backward: dd[p][c] = (d[p][c] > 0) sum_o dout[o][p] w[o][c];
// dw[o][c] += sum_p dout[o][p] d[p][c]; db[o] += sum_p dout[o][p]
template <int C>
__global__ void k_head_back(const float *dout, const bf16 *d, const float *w, bf16 *dd, float *dw,
                            float *db, int B, int HW) {
    __shared__ float red[4 * C];
    for (int i = threadIdx.x; i < 4 * C; i += blockDim.x) red[i] = 0.f;
    __syncthreads();
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float g[3] = {0.f, 0.f, 0.f};
    float lw[3][C];
    if (p < (long long)B * HW) {
        const long long n = p / HW, r = p - n * HW;
#pragma unroll
        for (int o = 0; o < 3; o++) g[o] = dout[(n * 3 + o) * HW + r];
#pragma unroll
        for (int c = 0; c < C; c++) {
            const float x = __bfloat162float(d[p * C + c]);
            const float v = g[0] * w[c] + g[1] * w[C + c] + g[2] * w[2 * C + c];
            dd[p * C + c] = __float2bfloat16(x > 0.f ? v : 0.f);
#pragma unroll
            for (int o = 0; o < 3; o++) lw[o][c] = g[o] * x;
        }
    } else {
#pragma unroll
        for (int o = 0; o < 3; o++)
#pragma unroll
            for (int c = 0; c < C; c++) lw[o][c] = 0.f;
    }
    // warp sums, then one shared atomic per warp and value
#pragma unroll
    for (int o = 0; o < 3; o++) {
#pragma unroll
        for (int c = 0; c < C; c++) {
            float v = lw[o][c];
            for (int s = 16; s > 0; s >>= 1) v += __shfl_down_sync(0xffffffffu, v, s);
            if ((threadIdx.x & 31) == 0) atomicAdd(&red[o * C + c], v);
        }
        float v = g[o];
        for (int s = 16; s > 0; s >>= 1) v += __shfl_down_sync(0xffffffffu, v, s);
        if ((threadIdx.x & 31) == 0) atomicAdd(&red[3 * C + o], v);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * C; i += blockDim.x) atomicAdd(dw + i, red[i]);
    if (threadIdx.x < 3) atomicAdd(db + threadIdx.x, red[3 * C + threadIdx.x]);
}

// db[c] += sum_p dz[p][c] (NHWC BF16), C <= 256
__global__ void k_colsum(const bf16 *dz, long long P, int C, float *db) {
    __shared__ float s[EW];
    const int c = threadIdx.x % C, rows = EW / C;
    const int r0 = threadIdx.x / C;
    float a = 0.f;
    if (r0 < rows)
        for (long long p = (long long)blockIdx.x * rows + r0; p < P; p += (long long)gridDim.x * rows)
            a += __bfloat162float(dz[p * C + c]);
    s[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x < C) {
        float t = 0.f;
        for (int r = 0; r < rows; r++) t += s[r * C + threadIdx.x];
        atomicAdd(db + threadIdx.x, t);
    }
}

// Adam on the flat FP32 master vector; refreshes the BF16 copies.
__global__ void k_adam(float *w, const float *g, float *m, float *v, bf16 *wb, long long n, float lr,
                       float c1, float c2) {
    const long long i = (long long)blockIdx.x * EW + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi, vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    w[i] = wi;
    wb[i] = __float2bfloat16(wi);
}

__global__ void k_to_bf16(const float *w, bf16 *wb, long long n) {
    const long long i = (long long)blockIdx.x * EW + threadIdx.x;
    if (i < n) wb[i] = __float2bfloat16(w[i]);
}

// wt[ci][tap][co] = w[co][tap][ci]
__global__ void k_transpose_w(const bf16 *w, bf16 *wt, int Co, int taps, int Ci) {
    const long long i = (long long)blockIdx.x * EW + threadIdx.x;
    if (i >= (long long)Co * taps * Ci) return;
    const int ci = (int)(i % Ci), tap = (int)((i / Ci) % taps), co = (int)(i / ((long long)Ci * taps));
    wt[((long long)ci * taps + tap) * Co + co] = w[i];
}

// network input of one case: mask (owner >= 0) and Re / 100, zero elsewhere
__global__ void k_case_input(const int32_t *owner, float re100, float *in, int HW) {
    const int i = blockIdx.x * EW + threadIdx.x;
    if (i >= HW) return;
    in[i] = owner[i] >= 0 ? 1.f : 0.f;
    in[HW + i] = re100;
    for (int c = 2; c < 8; c++) in[c * HW + i] = 0.f;
}

}  // namespace nn

// ================================================================ network

using nn::bf16;

namespace {

struct Conv {
    int ci, co, k;           // k = 3 or 1
    size_t w_off, b_off;     // into the flat parameter vector (internal layout)
    bf16 *wt = nullptr;      // transposed BF16 weights [ci][tap][co]
};

struct Level {
    int H, W, C;
    bf16 *inp = nullptr;  // pooled input (l > 0)
    bf16 *ea = nullptr, *e = nullptr;              // encoder: relu(conv a), level output
    bf16 *cat = nullptr, *da = nullptr, *d = nullptr;  // decoder (l < L-1)
    bf16 *g1 = nullptr, *g2 = nullptr, *gcat = nullptr, *gin = nullptr;  // gradients
};

}  // namespace

struct lbm_unet {
    lbm_unet_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<Conv> convs;  // parameter order
    std::vector<Level> lv;
    long long nparam = 0;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    bf16 *wb = nullptr;      // BF16 copy of the whole vector (biases unused)
    bf16 *x = nullptr;       // packed input [P0][8]
    float *out = nullptr, *dout = nullptr;
    float *io_in = nullptr, *io_out = nullptr, *io_tgt = nullptr, *io_fl = nullptr;  // staging
    float *grad_abi = nullptr;
    float *cnt = nullptr;
    double *loss = nullptr;
    int *err_d = nullptr;    // bit 0: a bounded wait of a tensor-core kernel ran out
    long long wait_limit = nn::TC_SPIN;  // polls of an mbarrier before a wait gives up
    int sms = 0;             // streaming multiprocessors of the device
    long long adam_t = 0;
    std::string err;
    std::vector<void *> allocs;
};

namespace {

thread_local std::string g_nn_error;

lbm_status nfail(lbm_unet *n, lbm_status st, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
lbm_status nfail(lbm_unet *n, lbm_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (n) n->err = buf;
    else g_nn_error = buf;
    return st;
}

#define NCK(n, call)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return nfail((n), e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,     \
                         "%s failed: %s", #call, cudaGetErrorString(e_));                  \
    } while (0)

// after a synchronisation: a tensor-core kernel that gave up waiting
lbm_status check_err(lbm_unet *n) {
    int e = 0;
    NCK(n, cudaMemcpyAsync(&e, n->err_d, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
    NCK(n, cudaStreamSynchronize(n->stream));
    if (e) {
        cudaMemsetAsync(n->err_d, 0, sizeof(int), n->stream);
        return nfail(n, LBM_ETIMEOUT, "a bounded wait of the tensor-core convolution ran out");
    }
    return LBM_OK;
}

template <class T>
cudaError_t nalloc(lbm_unet *n, T **p, size_t count) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T) + 16);
    if (e == cudaSuccess) n->allocs.push_back(*p);
    return e;
}

void nrelease(lbm_unet *n) {
    if (!n) return;
    for (void *p : n->allocs) cudaFree(p);
    if (n->own_stream && n->stream) cudaStreamDestroy(n->stream);
    delete n;
}

int conv_index(const lbm_unet *n, const char kind, int l, int ab) {
    // order: enc0a enc0b ... enc{L-1}b, dec{L-2}a dec{L-2}b ... dec0b, head
    const int L = n->cfg.levels;
    if (kind == 'e') return 2 * l + ab;
    if (kind == 'd') return 2 * L + 2 * (L - 2 - l) + ab;
    return 2 * L + 2 * (L - 1);
}

template <int BN>
cudaError_t launch_tc(lbm_unet *n, const nn::ConvOp &op) {
    constexpr int stages = nn::TC_STAGES * (nn::TC_M * nn::TC_K * 2 + BN * nn::TC_K * 2);
    const int table = ((op.K + nn::TC_K - 1) / nn::TC_K) * nn::TC_K;  // 8 bytes per 8 K elements
    if (table > nn::TC_TABLE_MAX) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(nn::k_conv_tc<BN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             stages + nn::TC_TABLE_MAX);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const dim3 grid((op.M + nn::TC_M - 1) / nn::TC_M, (op.N + BN - 1) / BN);
    nn::k_conv_tc<BN><<<grid, nn::TC_THREADS, stages + table, n->stream>>>(op, n->wait_limit, n->err_d);
    return cudaGetLastError();
}

// N tile: the output channels rounded up to 32 or 64, else 128 unless that
// leaves fewer than two tiles per SM
cudaError_t launch_conv_tc(lbm_unet *n, const nn::ConvOp &op) {
    const int mt = (op.M + nn::TC_M - 1) / nn::TC_M;
    if (op.N <= 32) return launch_tc<32>(n, op);
    if (op.N <= 64 || (long long)mt * ((op.N + 127) / 128) < 2LL * n->sms) return launch_tc<64>(n, op);
    return launch_tc<128>(n, op);
}

cudaError_t conv_fwd(lbm_unet *n, const Conv &cv, const bf16 *src, bf16 *dst, int B, int H, int W,
                     bool relu) {
    nn::ConvOp op{};
    op.src = src;
    op.w = n->wb + cv.w_off;
    op.bias = n->w + cv.b_off;
    op.mask = nullptr;
    op.out = dst;
    op.img = {B, H, W};
    op.Cs = cv.ci;
    op.taps = cv.k * cv.k;
    op.sign = 1;
    op.relu = relu;
    op.M = B * H * W;
    op.N = cv.co;
    op.K = op.taps * cv.ci;
    op.kchunk = op.K;
    return launch_conv_tc(n, op);
}

// gradient with respect to the conv's input (masked by mask > 0 when given)
cudaError_t conv_dgrad(lbm_unet *n, const Conv &cv, const bf16 *dz, const bf16 *mask, bf16 *dx,
                       int B, int H, int W) {
    nn::ConvOp op{};
    op.src = dz;
    op.w = cv.wt;
    op.bias = nullptr;
    op.mask = mask;
    op.out = dx;
    op.img = {B, H, W};
    op.Cs = cv.co;
    op.taps = cv.k * cv.k;
    op.sign = -1;
    op.relu = 0;
    op.M = B * H * W;
    op.N = cv.ci;
    op.K = op.taps * cv.co;
    op.kchunk = op.K;
    return launch_conv_tc(n, op);
}

template <int BN>
cudaError_t launch_wg(lbm_unet *n, const nn::WgradTc &op, int z) {
    constexpr int smem = nn::TC_STAGES * (nn::TC_M * nn::TC_K * 2 + BN * nn::TC_K * 2);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(nn::k_wgrad_tc<BN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const dim3 grid((op.M + nn::TC_M - 1) / nn::TC_M, (op.N + BN - 1) / BN, z);
    nn::k_wgrad_tc<BN><<<grid, nn::TC_THREADS, smem, n->stream>>>(op, n->wait_limit, n->err_d);
    return cudaGetLastError();
}

cudaError_t conv_wgrad(lbm_unet *n, const Conv &cv, const bf16 *dz, const bf16 *x, int B, int H,
                       int W) {
    if (cv.k == 3) {
        nn::WgradTc op{};
        op.dz = dz;
        op.x = x;
        op.dw = n->g + cv.w_off;
        op.img = {B, H, W};
        op.Co = cv.co;
        op.Ci = cv.ci;
        op.taps = 9;
        op.M = 9 * cv.ci;
        op.N = cv.co;
        op.K = B * H * W;
        const int bn = cv.co <= 32 ? 32 : (cv.co <= 64 ? 64 : 128);
        const int mt = (op.M + nn::TC_M - 1) / nn::TC_M, nt = (op.N + bn - 1) / bn;
        const int kt = (op.K + nn::TC_K - 1) / nn::TC_K;
        int z = 4 * n->sms / (mt * nt);
        if (z < 1) z = 1;
        if (z > kt) z = kt;
        op.kchunk = ((kt + z - 1) / z) * nn::TC_K;
        z = (op.K + op.kchunk - 1) / op.kchunk;
        cudaError_t e = bn == 32 ? launch_wg<32>(n, op, z)
                                 : (bn == 64 ? launch_wg<64>(n, op, z) : launch_wg<128>(n, op, z));
        if (e != cudaSuccess) return e;
        const long long P = op.K;
        int nb = (int)((P * cv.co + nn::EW - 1) / nn::EW);
        if (nb > 1024) nb = 1024;
        nn::k_colsum<<<nb, nn::EW, 0, n->stream>>>(dz, P, cv.co, n->g + cv.b_off);
        return cudaGetLastError();
    }
    nn::WgradOp op{};
    op.dz = dz;
    op.x = x;
    op.dw = n->g + cv.w_off;
    op.img = {B, H, W};
    op.Co = cv.co;
    op.Ci = cv.ci;
    op.taps = cv.k * cv.k;
    op.M = cv.co;
    op.N = op.taps * cv.ci;
    op.K = B * H * W;
    const int mt = (op.M + nn::BM - 1) / nn::BM, nt = (op.N + nn::BN - 1) / nn::BN;
    int z = 1200 / (mt * nt);
    const int kt = (op.K + nn::BK - 1) / nn::BK;
    if (z < 1) z = 1;
    if (z > kt) z = kt;
    op.kchunk = ((kt + z - 1) / z) * nn::BK;
    z = (op.K + op.kchunk - 1) / op.kchunk;
    const dim3 grid(mt, nt, z);
    nn::k_gemm<nn::WgradOp><<<grid, nn::GEMM_THREADS, 0, n->stream>>>(op);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long P = op.K;
    int nb = (int)((P * cv.co + nn::EW - 1) / nn::EW);
    if (nb > 1024) nb = 1024;
    nn::k_colsum<<<nb, nn::EW, 0, n->stream>>>(dz, P, cv.co, n->g + cv.b_off);
    return cudaGetLastError();
}

cudaError_t refresh_weights(lbm_unet *n) {
    nn::k_to_bf16<<<nn::blocks(n->nparam), nn::EW, 0, n->stream>>>(n->w, n->wb, n->nparam);
    cudaError_t e = cudaGetLastError();
    for (const Conv &cv : n->convs) {
        if (e != cudaSuccess) return e;
        const long long cnt = (long long)cv.co * cv.k * cv.k * cv.ci;
        nn::k_transpose_w<<<nn::blocks(cnt), nn::EW, 0, n->stream>>>(n->wb + cv.w_off, cv.wt, cv.co,
                                                                   cv.k * cv.k, cv.ci);
        e = cudaGetLastError();
    }
    return e;
}

lbm_status forward(lbm_unet *n, const float *in_dev, int B) {
    const int L = n->cfg.levels, H = n->cfg.height, W = n->cfg.width;
    NCK(n, (nn::k_pack_input<<<nn::blocks((long long)B * H * W * 8), nn::EW, 0, n->stream>>>(
               in_dev, n->x, B, H * W),
           cudaGetLastError()));
    for (int l = 0; l < L; l++) {
        Level &v = n->lv[l];
        const bf16 *inp = n->x;
        if (l > 0) {
            const Level &u = n->lv[l - 1];
            NCK(n, (nn::k_pool<<<nn::blocks((long long)B * v.H * v.W * u.C / 8), nn::EW, 0, n->stream>>>(
                       u.e, v.inp, B, u.H, u.W, u.C),
                   cudaGetLastError()));
            inp = v.inp;
        }
        NCK(n, conv_fwd(n, n->convs[conv_index(n, 'e', l, 0)], inp, v.ea, B, v.H, v.W, true));
        NCK(n, conv_fwd(n, n->convs[conv_index(n, 'e', l, 1)], v.ea, v.e, B, v.H, v.W, true));
    }
    const bf16 *d = n->lv[L - 1].e;
    for (int l = L - 2; l >= 0; l--) {
        Level &v = n->lv[l];
        const int Cu = n->lv[l + 1].C;
        NCK(n, (nn::k_upcat<<<nn::blocks((long long)B * v.H * v.W * (Cu + v.C) / 8), nn::EW, 0,
                              n->stream>>>(d, v.e, v.cat, B, v.H, v.W, Cu, v.C),
               cudaGetLastError()));
        NCK(n, conv_fwd(n, n->convs[conv_index(n, 'd', l, 0)], v.cat, v.da, B, v.H, v.W, true));
        NCK(n, conv_fwd(n, n->convs[conv_index(n, 'd', l, 1)], v.da, v.d, B, v.H, v.W, true));
        d = v.d;
    }
    const Conv &hd = n->convs[conv_index(n, 'h', 0, 0)];
    NCK(n, (nn::k_head<<<nn::blocks((long long)B * H * W), nn::EW, 0, n->stream>>>(
               d, n->w + hd.w_off, n->w + hd.b_off, n->out, B, H * W, n->lv[0].C),
           cudaGetLastError()));
    return LBM_OK;
}

lbm_status backward(lbm_unet *n, const float *tgt_dev, const float *fl_dev, int B) {
    const int L = n->cfg.levels, H = n->cfg.height, W = n->cfg.width;
    const long long HW = (long long)H * W;
    NCK(n, cudaMemsetAsync(n->g, 0, n->nparam * sizeof(float), n->stream));
    NCK(n, cudaMemsetAsync(n->cnt, 0, sizeof(float), n->stream));
    NCK(n, cudaMemsetAsync(n->loss, 0, sizeof(double), n->stream));
    NCK(n, (nn::k_count<<<256, nn::EW, 0, n->stream>>>(fl_dev, B * HW, n->cnt), cudaGetLastError()));
    NCK(n, (nn::k_loss<<<1024, nn::EW, 0, n->stream>>>(n->out, tgt_dev, fl_dev, n->cnt, n->dout,
                                                       n->loss, B, (int)HW),
           cudaGetLastError()));
    // head: gradient of d0 (masked by d0 > 0) into lv[0].g1
    Level &v0 = n->lv[0];
    const bf16 *d0 = L > 1 ? v0.d : v0.e;
    const Conv &hd = n->convs[conv_index(n, 'h', 0, 0)];
    const unsigned hb = nn::blocks(B * HW);
    if (v0.C == 32)
        nn::k_head_back<32><<<hb, nn::EW, 0, n->stream>>>(n->dout, d0, n->w + hd.w_off, v0.g1,
                                                          n->g + hd.w_off, n->g + hd.b_off, B, (int)HW);
    else if (v0.C == 16)
        nn::k_head_back<16><<<hb, nn::EW, 0, n->stream>>>(n->dout, d0, n->w + hd.w_off, v0.g1,
                                                          n->g + hd.w_off, n->g + hd.b_off, B, (int)HW);
    else
        nn::k_head_back<8><<<hb, nn::EW, 0, n->stream>>>(n->dout, d0, n->w + hd.w_off, v0.g1,
                                                         n->g + hd.w_off, n->g + hd.b_off, B, (int)HW);
    NCK(n, cudaGetLastError());
    // decoder: g1 of level l holds d(d_l) (masked)
    for (int l = 0; l < L - 1; l++) {
        Level &v = n->lv[l];
        const Conv &cb = n->convs[conv_index(n, 'd', l, 1)], &ca = n->convs[conv_index(n, 'd', l, 0)];
        NCK(n, conv_wgrad(n, cb, v.g1, v.da, B, v.H, v.W));
        NCK(n, conv_dgrad(n, cb, v.g1, v.da, v.g2, B, v.H, v.W));
        NCK(n, conv_wgrad(n, ca, v.g2, v.cat, B, v.H, v.W));
        NCK(n, conv_dgrad(n, ca, v.g2, v.cat, v.gcat, B, v.H, v.W));
        Level &u = n->lv[l + 1];
        NCK(n, (nn::k_up_back<<<nn::blocks((long long)B * u.H * u.W * u.C / 8), nn::EW, 0, n->stream>>>(
                   v.gcat, u.C + v.C, u.g1, B, u.H, u.W, u.C),
               cudaGetLastError()));
    }
    // encoder: g1 of level l holds d(e_l) (masked)
    for (int l = L - 1; l >= 0; l--) {
        Level &v = n->lv[l];
        const Conv &cb = n->convs[conv_index(n, 'e', l, 1)], &ca = n->convs[conv_index(n, 'e', l, 0)];
        const bf16 *inp = l > 0 ? v.inp : n->x;
        NCK(n, conv_wgrad(n, cb, v.g1, v.ea, B, v.H, v.W));
        NCK(n, conv_dgrad(n, cb, v.g1, v.ea, v.g2, B, v.H, v.W));
        NCK(n, conv_wgrad(n, ca, v.g2, inp, B, v.H, v.W));
        if (l == 0) break;
        NCK(n, conv_dgrad(n, ca, v.g2, nullptr, v.gin, B, v.H, v.W));
        Level &u = n->lv[l - 1];
        NCK(n, (nn::k_pool_back<<<nn::blocks((long long)B * u.H * u.W * u.C / 8), nn::EW, 0, n->stream>>>(
                   v.gin, u.e, u.gcat, v.C + u.C, v.C, u.g1, B, u.H, u.W, u.C),
               cudaGetLastError()));
    }
    return LBM_OK;
}

// host permutation between the ABI layout [co][ci][k][k] and the internal
// [co][tap][ci]
void abi_to_internal(const lbm_unet *n, const float *a, std::vector<float> &w) {
    w.assign(n->nparam, 0.f);
    size_t o = 0;
    for (const Conv &cv : n->convs) {
        const int t = cv.k * cv.k;
        for (int co = 0; co < cv.co; co++)
            for (int ci = 0; ci < cv.ci; ci++)
                for (int tap = 0; tap < t; tap++)
                    w[cv.w_off + ((size_t)co * t + tap) * cv.ci + ci] = a[o + ((size_t)co * cv.ci + ci) * t + tap];
        o += (size_t)cv.co * cv.ci * t;
        for (int co = 0; co < cv.co; co++) w[cv.b_off + co] = a[o + co];
        o += cv.co;
    }
}

void internal_to_abi(const lbm_unet *n, const float *w, float *a) {
    size_t o = 0;
    for (const Conv &cv : n->convs) {
        const int t = cv.k * cv.k;
        for (int co = 0; co < cv.co; co++)
            for (int ci = 0; ci < cv.ci; ci++)
                for (int tap = 0; tap < t; tap++)
                    a[o + ((size_t)co * cv.ci + ci) * t + tap] = w[cv.w_off + ((size_t)co * t + tap) * cv.ci + ci];
        o += (size_t)cv.co * cv.ci * t;
        for (int co = 0; co < cv.co; co++) a[o + co] = w[cv.b_off + co];
        o += cv.co;
    }
}

lbm_status stage_inputs(lbm_unet *n, const float *in, const float *tgt, const float *fl, int B,
                        int on_device, const float **din, const float **dtgt, const float **dfl) {
    const size_t HW = (size_t)n->cfg.height * n->cfg.width;
    if (on_device) {
        *din = in;
        if (dtgt) *dtgt = tgt;
        if (dfl) *dfl = fl;
        return LBM_OK;
    }
    NCK(n, cudaMemcpyAsync(n->io_in, in, (size_t)B * 8 * HW * sizeof(float), cudaMemcpyHostToDevice,
                           n->stream));
    *din = n->io_in;
    if (dtgt) {
        NCK(n, cudaMemcpyAsync(n->io_tgt, tgt, (size_t)B * 3 * HW * sizeof(float),
                               cudaMemcpyHostToDevice, n->stream));
        *dtgt = n->io_tgt;
    }
    if (dfl) {
        NCK(n, cudaMemcpyAsync(n->io_fl, fl, (size_t)B * HW * sizeof(float), cudaMemcpyHostToDevice,
                               n->stream));
        *dfl = n->io_fl;
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_unet_create(const lbm_unet_config *cfg, lbm_unet **out) {
    if (!cfg || !out) return nfail(nullptr, LBM_EINVAL, "null argument");
    *out = nullptr;
    const lbm_unet_config &c = *cfg;
    if (c.levels < 2 || c.levels > 4 || c.base < 8 || c.base % 8 || c.base > 64)
        return nfail(nullptr, LBM_EINVAL, "levels must be 2..4 and base a multiple of 8 up to 64");
    const int div = 1 << (c.levels - 1);
    if (c.height < div || c.width < div || c.height % div || c.width % div)
        return nfail(nullptr, LBM_EINVAL, "height and width must be multiples of %d", div);
    if (c.max_batch < 1 || (long long)c.max_batch * c.height * c.width >= (1ll << 31))
        return nfail(nullptr, LBM_EINVAL, "max_batch out of range");
    if (c.base != 8 && c.base != 16 && c.base != 32)
        return nfail(nullptr, LBM_EINVAL, "base must be 8, 16 or 32");
    if (cudaSetDevice(c.device) != cudaSuccess)
        return nfail(nullptr, LBM_ECUDA, "cannot select device %d", c.device);
    lbm_unet *n = new (std::nothrow) lbm_unet;
    if (!n) return nfail(nullptr, LBM_ENOMEM, "host allocation failed");
    n->cfg = c;
    if (cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, c.device) != cudaSuccess ||
        n->sms < 1)
        n->sms = 1;
    if (c.stream) {
        n->stream = static_cast<cudaStream_t>(c.stream);
    } else {
        if (cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking) != cudaSuccess) {
            nrelease(n);
            return nfail(nullptr, LBM_ECUDA, "stream creation failed");
        }
        n->own_stream = true;
    }
    const int L = c.levels;
    // parameter layout
    std::vector<int> ch(L);
    for (int l = 0; l < L; l++) ch[l] = c.base << l;
    size_t off = 0;
    auto add = [&](int ci, int co, int k) {
        Conv cv;
        cv.ci = ci;
        cv.co = co;
        cv.k = k;
        cv.w_off = off;
        off += (size_t)co * ci * k * k;
        off = (off + 7) & ~size_t(7);  // keep every weight block 16-byte aligned in BF16
        cv.b_off = off;
        off += (co + 7) & ~7;
        n->convs.push_back(cv);
    };
    int cin = 8;
    for (int l = 0; l < L; l++) {
        add(cin, ch[l], 3);
        add(ch[l], ch[l], 3);
        cin = ch[l];
    }
    for (int l = L - 2; l >= 0; l--) {
        add(ch[l + 1] + ch[l], ch[l], 3);
        add(ch[l], ch[l], 3);
    }
    add(ch[0], 3, 1);
    n->nparam = (long long)off;
    cudaError_t e = cudaSuccess;
    const size_t B = c.max_batch;
    e = nalloc(n, &n->w, off);
    if (e == cudaSuccess) e = nalloc(n, &n->g, off);
    if (e == cudaSuccess) e = nalloc(n, &n->m, off);
    if (e == cudaSuccess) e = nalloc(n, &n->v, off);
    if (e == cudaSuccess) e = nalloc(n, &n->wb, off);
    for (Conv &cv : n->convs)
        if (e == cudaSuccess) e = nalloc(n, &cv.wt, (size_t)cv.co * cv.ci * cv.k * cv.k);
    const size_t HW = (size_t)c.height * c.width;
    if (e == cudaSuccess) e = nalloc(n, &n->x, B * HW * 8);
    if (e == cudaSuccess) e = nalloc(n, &n->out, B * HW * 3);
    if (e == cudaSuccess) e = nalloc(n, &n->dout, B * HW * 3);
    if (e == cudaSuccess) e = nalloc(n, &n->io_in, B * HW * 8);
    if (e == cudaSuccess) e = nalloc(n, &n->io_out, B * HW * 3);
    if (e == cudaSuccess) e = nalloc(n, &n->io_tgt, B * HW * 3);
    if (e == cudaSuccess) e = nalloc(n, &n->io_fl, B * HW);
    if (e == cudaSuccess) e = nalloc(n, &n->cnt, 1);
    if (e == cudaSuccess) e = nalloc(n, &n->loss, 1);
    if (e == cudaSuccess) e = nalloc(n, &n->err_d, 1);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->err_d, 0, sizeof(int), n->stream);
    n->lv.resize(L);
    for (int l = 0; l < L && e == cudaSuccess; l++) {
        Level &v = n->lv[l];
        v.H = c.height >> l;
        v.W = c.width >> l;
        v.C = ch[l];
        const size_t P = B * v.H * v.W;
        const int cprev = l > 0 ? ch[l - 1] : 8;
        const int cnext = l + 1 < L ? ch[l + 1] : 0;
        if (l > 0) e = nalloc(n, &v.inp, P * cprev);
        if (e == cudaSuccess) e = nalloc(n, &v.ea, P * v.C);
        if (e == cudaSuccess) e = nalloc(n, &v.e, P * v.C);
        if (e == cudaSuccess && l < L - 1) e = nalloc(n, &v.cat, P * (v.C + cnext));
        if (e == cudaSuccess && l < L - 1) e = nalloc(n, &v.da, P * v.C);
        if (e == cudaSuccess && l < L - 1) e = nalloc(n, &v.d, P * v.C);
        if (e == cudaSuccess) e = nalloc(n, &v.g1, P * v.C);
        if (e == cudaSuccess) e = nalloc(n, &v.g2, P * v.C);
        if (e == cudaSuccess && l < L - 1) e = nalloc(n, &v.gcat, P * (v.C + cnext));
        if (e == cudaSuccess && l > 0) e = nalloc(n, &v.gin, P * cprev);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, off * sizeof(float), n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, off * sizeof(float), n->stream);
    if (e != cudaSuccess) {
        lbm_status st = e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
        nfail(nullptr, st, "lbm_unet_create: %s", cudaGetErrorString(e));
        nrelease(n);
        return st;
    }
    // He-normal weights (std sqrt(2 / fan_in)), zero biases, seeded
    std::vector<float> w(off, 0.f);
    std::mt19937_64 rng(c.seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    for (const Conv &cv : n->convs) {
        const double sd = std::sqrt(2.0 / (cv.ci * cv.k * cv.k));
        for (size_t i = 0; i < (size_t)cv.co * cv.ci * cv.k * cv.k; i++) w[cv.w_off + i] = (float)(sd * nd(rng));
    }
    e = cudaMemcpyAsync(n->w, w.data(), off * sizeof(float), cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) e = refresh_weights(n);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    if (e != cudaSuccess) {
        nfail(nullptr, LBM_ECUDA, "lbm_unet_create: %s", cudaGetErrorString(e));
        nrelease(n);
        return LBM_ECUDA;
    }
    *out = n;
    return LBM_OK;
}

lbm_status lbm_unet_destroy(lbm_unet *n) {
    if (!n) return LBM_OK;
    cudaSetDevice(n->cfg.device);
    cudaStreamSynchronize(n->stream);
    nrelease(n);
    return LBM_OK;
}

const char *lbm_unet_last_error(const lbm_unet *n) { return n ? n->err.c_str() : g_nn_error.c_str(); }

lbm_status lbm_unet_set_wait_limit(lbm_unet *n, int64_t polls) {
    if (!n || polls < 0) return LBM_EINVAL;
    n->wait_limit = (long long)polls;
    return LBM_OK;
}

int64_t lbm_unet_param_count(const lbm_unet *n) {
    if (!n) return -1;
    int64_t s = 0;
    for (const Conv &cv : n->convs) s += (int64_t)cv.co * cv.ci * cv.k * cv.k + cv.co;
    return s;
}

lbm_status lbm_unet_get_params(lbm_unet *n, float *a, int32_t on_device) {
    if (!n || !a) return LBM_EINVAL;
    NCK(n, cudaSetDevice(n->cfg.device));
    std::vector<float> w(n->nparam), h(lbm_unet_param_count(n));
    NCK(n, cudaMemcpyAsync(w.data(), n->w, w.size() * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    NCK(n, cudaStreamSynchronize(n->stream));
    internal_to_abi(n, w.data(), h.data());
    if (on_device) {
        NCK(n, cudaMemcpyAsync(a, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, n->stream));
        NCK(n, cudaStreamSynchronize(n->stream));
    } else {
        std::memcpy(a, h.data(), h.size() * sizeof(float));
    }
    return LBM_OK;
}

lbm_status lbm_unet_set_params(lbm_unet *n, const float *a, int32_t on_device) {
    if (!n || !a) return LBM_EINVAL;
    NCK(n, cudaSetDevice(n->cfg.device));
    std::vector<float> h(lbm_unet_param_count(n)), w;
    if (on_device) {
        NCK(n, cudaMemcpyAsync(h.data(), a, h.size() * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
        NCK(n, cudaStreamSynchronize(n->stream));
    } else {
        std::memcpy(h.data(), a, h.size() * sizeof(float));
    }
    for (float x : h)
        if (!std::isfinite(x)) return nfail(n, LBM_EINVAL, "non-finite parameter");
    abi_to_internal(n, h.data(), w);
    NCK(n, cudaMemcpyAsync(n->w, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice, n->stream));
    NCK(n, refresh_weights(n));
    NCK(n, cudaMemsetAsync(n->m, 0, n->nparam * sizeof(float), n->stream));
    NCK(n, cudaMemsetAsync(n->v, 0, n->nparam * sizeof(float), n->stream));
    n->adam_t = 0;
    NCK(n, cudaStreamSynchronize(n->stream));
    return LBM_OK;
}

lbm_status lbm_unet_forward(lbm_unet *n, const float *in, float *out, int32_t B, int32_t on_device) {
    if (!n || !in || !out || B < 1 || B > n->cfg.max_batch) return LBM_EINVAL;
    NCK(n, cudaSetDevice(n->cfg.device));
    const float *din = nullptr;
    lbm_status st = stage_inputs(n, in, nullptr, nullptr, B, on_device, &din, nullptr, nullptr);
    if (st == LBM_OK) st = forward(n, din, B);
    if (st != LBM_OK) return st;
    const size_t bytes = (size_t)B * 3 * n->cfg.height * n->cfg.width * sizeof(float);
    NCK(n, cudaMemcpyAsync(out, n->out, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           n->stream));
    if (!on_device) return check_err(n);
    return LBM_OK;
}

lbm_status lbm_unet_gradients(lbm_unet *n, const float *in, const float *tgt, const float *fl,
                              int32_t B, float *grads, double *loss, int32_t on_device) {
    if (!n || !in || !tgt || !fl || !grads || B < 1 || B > n->cfg.max_batch) return LBM_EINVAL;
    NCK(n, cudaSetDevice(n->cfg.device));
    const float *din, *dt, *df;
    lbm_status st = stage_inputs(n, in, tgt, fl, B, on_device, &din, &dt, &df);
    if (st == LBM_OK) st = forward(n, din, B);
    if (st == LBM_OK) st = backward(n, dt, df, B);
    if (st != LBM_OK) return st;
    std::vector<float> g(n->nparam), h(lbm_unet_param_count(n));
    double l = 0.0;
    NCK(n, cudaMemcpyAsync(g.data(), n->g, g.size() * sizeof(float), cudaMemcpyDeviceToHost, n->stream));
    NCK(n, cudaMemcpyAsync(&l, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    NCK(n, cudaStreamSynchronize(n->stream));
    st = check_err(n);
    if (st != LBM_OK) return st;
    internal_to_abi(n, g.data(), h.data());
    if (on_device) {
        NCK(n, cudaMemcpyAsync(grads, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, n->stream));
        NCK(n, cudaStreamSynchronize(n->stream));
    } else {
        std::memcpy(grads, h.data(), h.size() * sizeof(float));
    }
    if (loss) *loss = l;
    return LBM_OK;
}

lbm_status lbm_unet_train_step(lbm_unet *n, const float *in, const float *tgt, const float *fl,
                               int32_t B, float lr, double *loss, int32_t on_device) {
    if (!n || !in || !tgt || !fl || B < 1 || B > n->cfg.max_batch || !(lr > 0.f)) return LBM_EINVAL;
    NCK(n, cudaSetDevice(n->cfg.device));
    const float *din, *dt, *df;
    lbm_status st = stage_inputs(n, in, tgt, fl, B, on_device, &din, &dt, &df);
    if (st == LBM_OK) st = forward(n, din, B);
    if (st == LBM_OK) st = backward(n, dt, df, B);
    if (st != LBM_OK) return st;
    n->adam_t++;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)n->adam_t));
    const float c2 = (float)(1.0 - std::pow(0.999, (double)n->adam_t));
    NCK(n, (nn::k_adam<<<nn::blocks(n->nparam), nn::EW, 0, n->stream>>>(n->w, n->g, n->m, n->v, n->wb,
                                                                       n->nparam, lr, c1, c2),
           cudaGetLastError()));
    for (const Conv &cv : n->convs) {
        const long long cnt = (long long)cv.co * cv.k * cv.k * cv.ci;
        NCK(n, (nn::k_transpose_w<<<nn::blocks(cnt), nn::EW, 0, n->stream>>>(n->wb + cv.w_off, cv.wt, cv.co,
                                                                          cv.k * cv.k, cv.ci),
               cudaGetLastError()));
    }
    if (loss) {
        NCK(n, cudaMemcpyAsync(loss, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
        return check_err(n);
    }
    return LBM_OK;
}

lbm_status lbm_unet_input(lbm_unet *n, const int32_t *owner, double re, float *in) {
    if (!n || !owner || !in || !std::isfinite(re)) return LBM_EINVAL;
    NCK(n, cudaSetDevice(n->cfg.device));
    const int HW = n->cfg.height * n->cfg.width;
    NCK(n, (nn::k_case_input<<<nn::blocks(HW), nn::EW, 0, n->stream>>>(owner, (float)(re / 100.0), in, HW),
           cudaGetLastError()));
    return LBM_OK;
}

}  // extern "C"
