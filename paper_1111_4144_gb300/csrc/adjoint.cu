// Adjoint of the inverse on Hermitian matrices (not in the paper):
//   dA = -X S X,   S = (G + G^H) / 2,
// the gradient of a real loss L(X) with respect to a Hermitian A when
// X = A^{-1} and G = dL/dX.  It reuses the forward X (no refactorisation).
//
// One warp per matrix.  X (expanded from its stored upper half) and S are
// squares in shared memory; T = S X is formed column by column (lane j owns
// columns j and j+32), then the upper half of -X T, mirrored to keep dA
// exactly Hermitian.
#include <algorithm>
#include <mutex>

#include "batched.cuh"
#include "dispatch.h"

namespace cholinv {

template <typename V>
CHOL_HD size_t bwd_warp_bytes(int N) {
    const size_t b = (size_t)3 * N * (N + 1) * sizeof(V);
    return (b + 15) / 16 * 16;
}

template <typename V>
__global__ void k_backward(BwdParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = p.max_n;
    const int LD = N + 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    V* Xf = reinterpret_cast<V*>(smem_raw + (size_t)w * bwd_warp_bytes<V>(N));
    V* Sf = Xf + (size_t)N * LD;
    V* Tf = Sf + (size_t)N * LD;
    const V* X = static_cast<const V*>(p.X);
    const V* G = static_cast<const V*>(p.G);
    V* dA = static_cast<V*>(p.dA);

    for (int b = blockIdx.x * wpc + w; b < p.batch; b += gridDim.x * wpc) {
        const int n = p.n ? p.n[b] : N;
        if (n <= 0 || n > N) continue;
        const int64_t og = p.off ? p.off[b] : (int64_t)b * N * N;
        const int64_t ox = p.xoff ? p.xoff[b] : (int64_t)b * (p.layout ? tri64(N) : (int64_t)N * N);
        for (int i = 0; i < n; ++i)
            for (int j = i + lane; j < n; j += 32) {
                const int64_t gx = p.layout ? (int64_t)pidx(n, i, j) : (int64_t)i * n + j;
                V x = X[ox + gx];
                if (i == j) x = from_real<V>(re_of(x));
                Xf[i * LD + j] = x;
                Xf[j * LD + i] = conj_v(x);
                // S = (G + G^H)/2
                const V gij = G[og + (int64_t)i * n + j], gji = G[og + (int64_t)j * n + i];
                using R = typename traits<V>::real;
                const V sij = scale_v(gij + conj_v(gji), R(0.5));
                Sf[i * LD + j] = (i == j) ? from_real<V>(re_of(sij)) : sij;
                Sf[j * LD + i] = conj_v(sij);
            }
        __syncwarp();
        // T = S X
        for (int j = lane; j < n; j += 32)
            for (int i = 0; i < n; ++i) {
                V acc = zero_v<V>();
                for (int k = 0; k < n; ++k) acc = fma_v(Sf[i * LD + k], Xf[k * LD + j], acc);
                Tf[i * LD + j] = acc;
            }
        __syncwarp();
        // dA = -X T (upper half computed, mirrored)
        for (int j = lane; j < n; j += 32)
            for (int i = 0; i <= j; ++i) {
                V acc = zero_v<V>();
                for (int k = 0; k < n; ++k) acc = fma_v(Xf[i * LD + k], Tf[k * LD + j], acc);
                V d = zero_v<V>() - acc;
                if (i == j) d = from_real<V>(re_of(d));
                if (p.flags & CHOL_FLAG_GRAD_UPPER) {
                    using R = typename traits<V>::real;
                    dA[og + (int64_t)i * n + j] = (i == j) ? d : scale_v(d, R(2));
                    if (i != j) dA[og + (int64_t)j * n + i] = zero_v<V>();
                } else {
                    dA[og + (int64_t)i * n + j] = d;
                    if (i != j) dA[og + (int64_t)j * n + i] = conj_v(d);
                }
            }
        __syncwarp();
    }
}

template <typename V>
static cudaError_t launch_bwd_t(const BwdParams& p, cudaStream_t s, bool dry) {
    static std::once_flag once;
    static cudaError_t setup = cudaSuccess;
    std::call_once(once, [&] {
        setup = cudaFuncSetAttribute(k_backward<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    if (setup != cudaSuccess || dry) return setup;
    const size_t per = bwd_warp_bytes<V>(p.max_n);
    const int warps = (int)std::max<size_t>(1, std::min<size_t>(4, 98304 / per));
    int per_sm = 1;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_backward<V>, 32 * warps, per * warps);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min((p.batch + warps - 1) / warps, device_info().sms * std::max(per_sm, 1)));
    k_backward<V><<<grid, 32 * warps, per * warps, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_backward(int dtype, const BwdParams& p, cudaStream_t s, bool dry) {
    switch (dtype) {
        case CHOL_F32: return launch_bwd_t<float>(p, s, dry);
        case CHOL_F64: return launch_bwd_t<double>(p, s, dry);
        case CHOL_C64: return launch_bwd_t<cpx<float>>(p, s, dry);
        case CHOL_C128: return launch_bwd_t<cpx<double>>(p, s, dry);
    }
    return cudaErrorInvalidValue;
}

}  // namespace cholinv
