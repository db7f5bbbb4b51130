// Tensor-core GEMM for the blocked path on sm_103a (tcgen05 + TMA + TMEM):
//   C = alpha * A B^T + beta * C     (or one K-slice of A B^T into partial[z])
// A is M x K and B is N x K, both K-major FP32 in global memory, read through
// TMA tensor maps in 128 x 32 tiles with the 128-byte swizzle into a
// multi-stage shared-memory ring; one elected thread issues
// tcgen05.mma.kind::tf32 (M = 128, N = 128, K = 8 per instruction) into a
// 128 x 128 FP32 accumulator in tensor memory; four warps read it back with
// tcgen05.ld for the epilogue.
//
// split3 = 1 forms each product as three TF32 products (Ootomo & Yokota's
// error-corrected TF32, 2022): with x_hi = tf32(x) and x_lo = tf32(x - x_hi)
// (both rounded to nearest), A B^T ~ A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T,
// accurate to about FP32 (single-pass TF32 keeps only 11 significant bits).
// Two converter warps split each tile in shared memory after it lands.
//
// With CPRE (beta != 0, no split-K), the producer also fetches the C tile
// with bulk asynchronous copies (one per row) before the main loop, so that
// the read half of the read-modify-write overlaps the products.
//
// Every wait on an mbarrier is bounded (about one second); on expiry the
// kernel records an error, stops issuing work, waits (bounded) for what it
// issued, frees its tensor memory and returns.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace cholinv {
namespace umma {

constexpr int BM = 128, BN = 128, BK = 32;
constexpr int TILE_FLOATS = BM * BK;  // == BN * BK
constexpr int THREADS = 128;

CHOL_D uint32_t sa(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
CHOL_D uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
CHOL_D void mbar_init(uint64_t* b, uint32_t c) {
    asm volatile("mbarrier.init.shared.b64 [%0], %1;" ::"r"(sa(b)), "r"(c) : "memory");
}
CHOL_D void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(sa(b)), "r"(bytes)
                 : "memory");
}
CHOL_D void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(sa(b)) : "memory");
}
CHOL_D bool mbar_try(uint64_t* b, uint32_t par) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(sa(b)), "r"(par)
        : "memory");
    return ok != 0;
}
// Bounded wait: false (and *err set) after about one second, or at once if
// another thread already gave up.
CHOL_D bool mbar_wait(uint64_t* b, uint32_t par, int* err) {
    const uint64_t t0 = gtimer();
    while (!mbar_try(b, par)) {
        if (*reinterpret_cast<volatile int*>(err)) return false;
        if (gtimer() - t0 > 1000000000ull) {
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}
// Bounded wait that reports nothing (used while draining after a give-up).
CHOL_D bool mbar_wait_quiet(uint64_t* b, uint32_t par) {
    const uint64_t t0 = gtimer();
    while (!mbar_try(b, par))
        if (gtimer() - t0 > 1000000000ull) return false;
    return true;
}
CHOL_D void tma2d(void* dst, const CUtensorMap* m, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(sa(dst)),
        "l"(m), "r"(x), "r"(y), "r"(sa(bar))
        : "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (the layout the 128B-swizzled TMA tile has).
CHOL_D uint64_t sdesc(const void* p) {
    const uint64_t addr = sa(p);
    uint64_t d = (addr & 0x3FFFF) >> 4;   // start address
    d |= (uint64_t)1 << 16;               // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset
    d |= (uint64_t)1 << 46;               // descriptor version
    d |= (uint64_t)2 << 61;               // 128-byte swizzle
    return d;
}
// Instruction descriptor: D F32, A/B TF32, both K-major, N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

CHOL_D void mma_tf32(uint32_t dt, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(dt),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}
// Round to the nearest TF32 value (10 explicit mantissa bits), as an FP32 bit pattern.
CHOL_D float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
// One bulk asynchronous copy global -> shared (16-byte aligned, size a multiple of 16).
CHOL_D void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sa(dst)),
                 "l"(src), "r"(bytes), "r"(sa(bar))
                 : "memory");
}
CHOL_D void commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sa(b)) : "memory");
}

struct GemmArgs {
    int M, N, K;          // C is M x N; K summed
    int ax, ay, bx, by;   // tensor-map coordinates of A(0,0) and B(0,0) (x = K index)
    float alpha, beta;
    float* C;
    int64_t ldc;
    int upper;            // only entries with row <= col (tiles wholly below skipped)
    int kchunk;           // K per blockIdx.z
    float* partial;       // if set: raw slice products, [z][M][N]
    int split3;           // three-product TF32 split
    int* err;
};

template <int STAGES, int SPLIT3, int CPRE>
constexpr size_t smem_bytes() {
    return (size_t)STAGES * (SPLIT3 ? 4 : 2) * TILE_FLOATS * 4 + (CPRE ? (size_t)BM * BN * 4 : 0) + 1024 + 512;
}

template <int STAGES, int SPLIT3, int CPRE>
__global__ void __launch_bounds__(THREADS) k_umma_gemm(const __grid_constant__ CUtensorMap ta,
                                                        const __grid_constant__ CUtensorMap tb, GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    constexpr int TILES = SPLIT3 ? 4 : 2;  // A, B (, A_lo, B_lo) per stage
    float* ring = reinterpret_cast<float*>(sm);
    float* cbuf = ring + (size_t)STAGES * TILES * TILE_FLOATS;  // [BM][BN] C tile (CPRE)
    uint64_t* full = reinterpret_cast<uint64_t*>(cbuf + (CPRE ? BM * BN : 0));
    uint64_t* conv = full + STAGES;
    uint64_t* empty = conv + STAGES;
    uint64_t* done = empty + STAGES;
    uint64_t* cbar = done + 1;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(cbar + 1);
    const bool cpre = CPRE && g.beta != 0.f && g.partial == nullptr;
    auto tile = [&](int s, int which) { return ring + ((size_t)s * TILES + which) * TILE_FLOATS; };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (g.upper && m0 > n0 + BN - 1) return;  // uniform across the CTA: before any barrier or allocation
    const int kb = blockIdx.z * g.kchunk;
    const int ke = min(g.K, kb + g.kchunk);
    const int KT = ke > kb ? (ke - kb + BK - 1) / BK : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&conv[s], 64);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        mbar_init(cbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(tslot)), "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = *tslot;
    int issued = 0;  // k-tiles whose loads were issued (producer)

    const int crows = min(BM, g.M - m0);
    const uint32_t cbytes = (uint32_t)min(BN, g.N - n0) * 4u;
    if (warp == 0) {
        if (lane == 0) {
            if (cpre) {
                // the C tile, row by row, behind the products
                mbar_expect_tx(cbar, (uint32_t)crows * cbytes);
                for (int r = 0; r < crows; ++r)
                    bulk_g2s(cbuf + r * BN, g.C + (int64_t)(m0 + r) * g.ldc + n0, cbytes, cbar);
            }
            for (int kt = 0; kt < KT; ++kt) {
                const int s = kt % STAGES;
                if (kt >= STAGES && !mbar_wait(&empty[s], ((kt / STAGES) & 1) ^ 1, g.err)) break;
                mbar_expect_tx(&full[s], 2 * TILE_FLOATS * 4);
                const int kx = kb + kt * BK;
                tma2d(tile(s, 0), &ta, g.ax + kx, g.ay + m0, &full[s]);
                tma2d(tile(s, 1), &tb, g.bx + kx, g.by + n0, &full[s]);
                ++issued;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            for (int kt = 0; kt < KT; ++kt) {
                const int s = kt % STAGES;
                if (!mbar_wait(SPLIT3 ? &conv[s] : &full[s], (kt / STAGES) & 1, g.err)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int kk = 0; kk < BK / 8; ++kk) {
                    const uint64_t off = (uint64_t)((kk * 32) >> 4);
                    const uint64_t a = sdesc(tile(s, 0)) + off, b = sdesc(tile(s, 1)) + off;
                    const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
                    if (SPLIT3) {
                        const uint64_t al = sdesc(tile(s, 2)) + off, bl = sdesc(tile(s, 3)) + off;
                        mma_tf32(tbase, al, b, acc);  // small terms first
                        mma_tf32(tbase, a, bl, 1u);
                        mma_tf32(tbase, a, b, 1u);
                    } else {
                        mma_tf32(tbase, a, b, acc);
                    }
                }
                commit(&empty[s]);
            }
            commit(done);
        }
    } else if (SPLIT3) {
        // converters (warps 2, 3): x -> x_hi = tf32(x) (in place) and x_lo = tf32(x - x_hi)
        const int ct = threadIdx.x - 64;
        for (int kt = 0; kt < KT; ++kt) {
            const int s = kt % STAGES;
            if (!mbar_wait(&full[s], (kt / STAGES) & 1, g.err)) break;
#pragma unroll
            for (int w = 0; w < 2; ++w) {
                float4* src = reinterpret_cast<float4*>(tile(s, w));
                float4* lo = reinterpret_cast<float4*>(tile(s, 2 + w));
                for (int i = ct; i < TILE_FLOATS / 4; i += 64) {
                    float4 v = src[i], h, l;
                    h.x = to_tf32(v.x); l.x = to_tf32(v.x - h.x);
                    h.y = to_tf32(v.y); l.y = to_tf32(v.y - h.y);
                    h.z = to_tf32(v.z); l.z = to_tf32(v.z - h.z);
                    h.w = to_tf32(v.w); l.w = to_tf32(v.w - h.w);
                    src[i] = h;
                    lo[i] = l;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
            mbar_arrive(&conv[s]);
        }
    }
    __syncwarp();
    // Epilogue.  Warp w reads TMEM lanes 32w..32w+31 (rows m0 + 32w + lane)
    // into a shared-memory tile (the ring is idle once every MMA has
    // completed); the CTA then reads and writes C along rows, coalesced.
    int mine = KT == 0 ? 1 : (int)mbar_wait(done, 0, g.err);
    if (cpre && mine) mine = (int)mbar_wait(cbar, 0, g.err);
    const bool ok = __syncthreads_and(mine) != 0;
    if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        constexpr int LDS = BN + 1;  // row stride of the staging tile: conflict-free both ways
        float* stage = ring;
        const int rl = warp * 32 + lane;
        for (int c = 0; c < BN; c += 16) {
            uint32_t r[16];
            if (KT > 0) {
                const uint32_t taddr = tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15])
                    : "r"(taddr)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) r[i] = 0u;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) stage[rl * LDS + c + i] = __uint_as_float(r[i]);
        }
        __syncthreads();
        static_assert(THREADS == BN, "one thread per column of the tile");
        const int col = n0 + (int)threadIdx.x;
#pragma unroll 4
        for (int rr = 0; rr < BM; ++rr) {
            const int row = m0 + rr;
            if (row < g.M && col < g.N && !(g.upper && row > col)) {
                const float v = stage[rr * LDS + threadIdx.x];
                if (g.partial) {
                    g.partial[((int64_t)blockIdx.z * g.M + row) * g.N + col] = v;
                } else {
                    float o = g.alpha * v;
                    if (g.beta != 0.f) {
                        const float c0 = cpre ? cbuf[rr * BN + threadIdx.x] : g.C[(int64_t)row * g.ldc + col];
                        o = fmaf(g.beta, c0, o);
                    }
                    g.C[(int64_t)row * g.ldc + col] = o;
                }
            }
        }
    } else if (warp == 0 && lane == 0) {
        // gave up: let the loads already issued land before the shared memory is released
        for (int kt = 0; kt < issued; ++kt) mbar_wait_quiet(&full[kt % STAGES], (kt / STAGES) & 1);
        if (cpre) mbar_wait_quiet(cbar, 0);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(BN) : "memory");
}

}  // namespace umma
}  // namespace cholinv
