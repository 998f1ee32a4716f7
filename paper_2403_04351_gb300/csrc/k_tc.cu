// Complex GEMM on the sm_103a tensor cores: C = op(A) X in a split-BF16 form.
//
// The complex product is written as one real GEMM (complex as real
// sub-GEMMs): with A^ = [Re A | Im A] (K-major) and, for column n of X,
// B^ rows [Re X_n | -Im X_n] (giving Re C) and [Im X_n | Re X_n] (giving Im C),
// D = A^ B^^T holds [Re C | Im C].  Each real operand is split into a bf16
// high part and a bf16 remainder, and the three products hi.hi + hi.lo +
// lo.hi are accumulated in FP32 by running the K loop over three segments
// (A: hi, hi, lo; B: hi, lo, hi).  The products use tcgen05.mma (kind::f16,
// bf16 inputs, FP32 accumulator in tensor memory) on operands staged in
// shared memory by TMA (cp.async.bulk.tensor, 128-byte swizzle, K-major),
// issued by one thread through a four-stage mbarrier pipeline; every wait
// is bounded and raises flag bit 3 instead of hanging.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "rtd.h"
#include "rttddft.h"

#define TC_BM 128
#define TC_BK 64  // bf16 per K block = 128 bytes, one swizzle row
#define TC_STAGES 4

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(phase)
        : "memory");
    return ok != 0;
}
// bounded wait on an mbarrier phase: false after about 2^31 SM cycles (~1 s)
__device__ bool mbar_wait(uint64_t* b, uint32_t phase) {
    const long long t0 = clock64();
    while (!mbar_try_wait(b, phase))
        if (clock64() - t0 > (1ll << 31)) return false;
    return true;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)tm), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 B apart
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                  // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
    d |= (uint64_t)1 << 46;                  // descriptor version
    d |= (uint64_t)2 << 61;                  // 128-byte swizzle
    return d;
}
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[split][m][n] (FP32, row-major M x N) = sum over this split's K blocks
// of A^ B^^T; grid (M tiles, K splits, N tiles).
template <int NT>
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
              const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl, int nkb2,
              int kb_per_split, float* __restrict__ D, int M, int N, int* flag) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int A_BYTES = TC_BM * TC_BK * 2;
    constexpr int B_BYTES = NT * TC_BK * 2;
    constexpr int STAGE = A_BYTES + B_BYTES;
    constexpr uint32_t NCOLS = NT <= 32 ? 32 : (NT <= 64 ? 64 : (NT <= 128 ? 128 : 256));
    __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.z * NT;
    const int total = 3 * nkb2;
    const int kb0 = blockIdx.y * kb_per_split;
    const int kb1 = min(total, kb0 + kb_per_split);
    const int nk = kb1 - kb0;
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(NCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    // kind::f16 instruction descriptor: FP32 accumulator, bf16 A and B, both
    // K-major, N >> 3 at bit 17, M >> 4 at bit 24
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                           ((uint32_t)(TC_BM >> 4) << 24);
    if (tid == 0 && nk > 0) {
        int issued = 0;
        auto load = [&](int j) {
            const int kb = kb0 + j;
            const int s = j % TC_STAGES;
            const int seg = kb / nkb2, kx = (kb % nkb2) * TC_BK;
            unsigned char* sa = smem + s * STAGE;
            unsigned char* sb = sa + A_BYTES;
            mbar_expect_tx(&full[s], STAGE);
            tma_load_2d(sa, seg < 2 ? &tmAh : &tmAl, kx, m0, &full[s]);
            tma_load_2d(sb, seg == 1 ? &tmBl : &tmBh, kx, n0, &full[s]);
            issued = j + 1;
        };
        const int pre = nk < TC_STAGES ? nk : TC_STAGES;
        for (int j = 0; j < pre; ++j) load(j);
        bool ok = true;
        int consumed = 0;
        for (int j = 0; j < nk; ++j) {
            const int s = j % TC_STAGES;
            if (!mbar_wait(&full[s], (uint32_t)((j / TC_STAGES) & 1))) {
                ok = false;
                break;
            }
            consumed = j + 1;
            tc_fence_after();
            const uint32_t a0 = smem_u32(smem + s * STAGE), b0 = a0 + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk)
                umma_bf16(tmem, umma_desc(a0 + kk * 32), umma_desc(b0 + kk * 32), idesc, (j > 0 || kk > 0) ? 1u : 0u);
            umma_commit(&empty[s]);
            // refill the slot of the previous block once its products are done,
            // so that block j's products stay queued meanwhile
            const int jp = j - 1;
            if (jp >= 0 && jp + TC_STAGES < nk) {
                if (!mbar_wait(&empty[jp % TC_STAGES], (uint32_t)((jp / TC_STAGES) & 1))) {
                    ok = false;
                    break;
                }
                load(jp + TC_STAGES);
            }
        }
        umma_commit(&done);
        if (!ok) {
            abort_flag = 1;
            atomicOr(flag, 8);
            // let the copies already issued land before the block's shared memory goes away
            for (int j = consumed; j < issued; ++j) mbar_wait(&full[j % TC_STAGES], (uint32_t)((j / TC_STAGES) & 1));
        }
    }
    __syncthreads();
    const bool okd = (nk > 0) ? mbar_wait(&done, 0) : true;
    tc_fence_after();
    if (okd && !abort_flag && nk > 0) {
        const int row = m0 + warp * 32 + lane;
        float* drow = D + ((size_t)blockIdx.y * M + row) * N;
#pragma unroll 1
        for (int c = 0; c < NT; c += 8) {
            uint32_t r[8];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int col = n0 + c + q;
                    if (col < N) drow[col] = __uint_as_float(r[q]);
                }
            }
        }
    } else if (tid == 0 && !okd) {
        atomicOr(flag, 8);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS) : "memory");
}

// ------------------------------------------------------------ operand packing
__device__ __forceinline__ void split_bf16(double v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __double2bfloat16(v);
    lo = __double2bfloat16(v - (double)__bfloat162float(hi));
}

// A^ rows r < R (K-major, Kp columns): [Re v | Im v | 0 pad], v = A[r, k]
// (mode 0) or conj(A[k, r]) (mode 1), A complex column-major with ld.
__global__ void k_tc_pack_a(const zd* __restrict__ A, int ld, int R, int K, int Kp, int mode,
                            __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
    const size_t e = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (e >= (size_t)R * Kp) return;
    const int r = (int)(e / Kp), kp = (int)(e % Kp);
    double v = 0.0;
    if (kp < 2 * K) {
        const int k = kp < K ? kp : kp - K;
        const zd a = (mode == 0) ? A[r + (size_t)k * ld] : zconj(A[k + (size_t)r * ld]);
        v = (kp < K) ? a.x : a.y;
    }
    split_bf16(v, hi[e], lo[e]);
}

// B^ rows n' < Rp (K-major, Kp columns) from X (K x N complex, column-major):
// n' < N: [Re X_n | -Im X_n], N <= n' < 2N: [Im X_n | Re X_n], else 0.
__global__ void k_tc_pack_b(const zd* __restrict__ X, int ldx, int K, int N, int Kp, int Rp,
                            __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
    const size_t e = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (e >= (size_t)Rp * Kp) return;
    const int r = (int)(e / Kp), kp = (int)(e % Kp);
    double v = 0.0;
    if (r < 2 * N && kp < 2 * K) {
        const int n = r < N ? r : r - N;
        const int k = kp < K ? kp : kp - K;
        const zd x = X[k + (size_t)n * ldx];
        if (r < N) v = (kp < K) ? x.x : -x.y;
        else v = (kp < K) ? x.y : x.x;
    }
    split_bf16(v, hi[e], lo[e]);
}

// C[m, n] (+)= sum_s D[s][m][n] + i D[s][m][N + n]  (FP64 sums)
__global__ void k_tc_combine(const float* __restrict__ D, int splits, int M, int Nc, int Dn, zd* __restrict__ C,
                             int ldc, int beta_add) {
    const int e = blockIdx.x * 256 + threadIdx.x;
    if (e >= M * Nc) return;
    const int m = e % M, n = e / M;
    double re = 0.0, im = 0.0;
    for (int s = 0; s < splits; ++s) {
        const float* d = D + ((size_t)s * M + m) * Dn;
        re += (double)d[n];
        im += (double)d[Nc + n];
    }
    zd* c = C + m + (size_t)n * ldc;
    *c = beta_add ? zadd(*c, zmk(re, im)) : zmk(re, im);
}

// ------------------------------------------------------------ host side
typedef CUresult (*encode_fn_t)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static encode_fn_t get_encode() {
    static encode_fn_t fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (encode_fn_t)p;
    }
    return fn;
}

// 2-D bf16 tensor map, rows of `inner` elements (row pitch `pitch_elems`),
// box of 64 x box_rows elements, 128-byte swizzle
static int tc_tmap(CUtensorMap* tm, const void* base, uint64_t inner, uint64_t rows, uint64_t pitch_elems,
                   uint32_t box_rows) {
    encode_fn_t enc = get_encode();
    if (!enc) return -1;
    if (((uintptr_t)base & 15) || ((pitch_elems * 2) & 15)) return -2;
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {pitch_elems * 2};
    cuuint32_t box[2] = {TC_BK, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -3;
}

template <int NT>
static int tc_launch(const CUtensorMap& ah, const CUtensorMap& al, const CUtensorMap& bh, const CUtensorMap& bl,
                     int nkb2, int kbs, dim3 grid, float* D, int M, int N, int* flag, cudaStream_t s) {
    const size_t smem = 1024 + (size_t)TC_STAGES * (TC_BM * TC_BK * 2 + NT * TC_BK * 2);
    if (cudaFuncSetAttribute(k_tc_gemm<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    k_tc_gemm<NT><<<grid, 128, smem, s>>>(ah, al, bh, bl, nkb2, kbs, D, M, N, flag);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// One split-BF16 complex GEMM C = op(A) X (A: M x K for op N, K x M for op C;
// X: K x N; all complex FP64 column-major on the device), with its own
// workspace.  Returns an RTTDDFT_* code; synchronizes the stream.
int tc_zgemm(int opA, int M, int N, int K, const zd* A, int lda, const zd* X, int ldx, zd* C, int ldc,
             int beta_add, cudaStream_t s) {
    if (M < 0 || N < 0 || K < 0 || (opA != 0 && opA != 1)) return RTTDDFT_ERR_ARG;
    if (M == 0 || N == 0) return RTTDDFT_OK;
    if (K == 0) return RTTDDFT_ERR_ARG;
    if (lda < (opA ? K : M) || ldx < K || ldc < M || !A || !X || !C) return RTTDDFT_ERR_ARG;
    if (!get_encode()) return RTTDDFT_ERR_UNSUPPORTED;
    const int Kp = ((2 * K + TC_BK - 1) / TC_BK) * TC_BK;
    const int nkb2 = Kp / TC_BK;
    const int Dn = 2 * N;  // real columns of D
    int NT = ((Dn + 15) / 16) * 16;
    if (NT > 256) NT = 256;
    const int ntile = (Dn + NT - 1) / NT;
    const int Rp = ntile * NT;  // packed B rows (padded)
    const int mt = (M + TC_BM - 1) / TC_BM;
    const int total = 3 * nkb2;
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int splits = (2 * nsm + mt * ntile - 1) / (mt * ntile);
    splits = std::max(1, std::min(splits, std::max(1, total / 4)));
    const int kbs = (total + splits - 1) / splits;
    splits = (total + kbs - 1) / kbs;
    const size_t mrows = (size_t)mt * TC_BM;
    __nv_bfloat16 *ah = nullptr, *al = nullptr, *bh = nullptr, *bl = nullptr;
    float* D = nullptr;
    int* flag = nullptr;
    int rc = RTTDDFT_OK;
    if (cudaMalloc(&ah, mrows * Kp * 2) != cudaSuccess || cudaMalloc(&al, mrows * Kp * 2) != cudaSuccess ||
        cudaMalloc(&bh, (size_t)Rp * Kp * 2) != cudaSuccess || cudaMalloc(&bl, (size_t)Rp * Kp * 2) != cudaSuccess ||
        cudaMalloc(&D, (size_t)splits * M * Dn * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&flag, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        rc = RTTDDFT_ERR_OOM;
    }
    if (rc == RTTDDFT_OK) {
        cudaMemsetAsync(flag, 0, sizeof(int), s);
        cudaMemsetAsync(ah, 0, mrows * Kp * 2, s);
        cudaMemsetAsync(al, 0, mrows * Kp * 2, s);
        k_tc_pack_a<<<(unsigned)(((size_t)M * Kp + 255) / 256), 256, 0, s>>>(A, lda, M, K, Kp, opA, ah, al);
        k_tc_pack_b<<<(unsigned)(((size_t)Rp * Kp + 255) / 256), 256, 0, s>>>(X, ldx, K, N, Kp, Rp, bh, bl);
        CUtensorMap tah, tal, tbh, tbl;
        if (tc_tmap(&tah, ah, Kp, mrows, Kp, TC_BM) || tc_tmap(&tal, al, Kp, mrows, Kp, TC_BM) ||
            tc_tmap(&tbh, bh, Kp, Rp, Kp, NT) || tc_tmap(&tbl, bl, Kp, Rp, Kp, NT)) {
            rc = RTTDDFT_ERR_CUDA;
        } else {
            dim3 grid(mt, splits, ntile);
            int lr = 0;
            switch (NT) {
#define RTD_TC(n) \
    case n: lr = tc_launch<n>(tah, tal, tbh, tbl, nkb2, kbs, grid, D, M, Dn, flag, s); break;
                RTD_TC(16) RTD_TC(32) RTD_TC(48) RTD_TC(64) RTD_TC(80) RTD_TC(96) RTD_TC(112) RTD_TC(128)
                RTD_TC(144) RTD_TC(160) RTD_TC(176) RTD_TC(192) RTD_TC(208) RTD_TC(224) RTD_TC(240) RTD_TC(256)
#undef RTD_TC
                default: lr = -1;
            }
            if (lr) rc = RTTDDFT_ERR_CUDA;
            else k_tc_combine<<<(M * N + 255) / 256, 256, 0, s>>>(D, splits, M, N, Dn, C, ldc, beta_add);
        }
    }
    int hflag = 0;
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = RTTDDFT_ERR_CUDA;
    if (rc == RTTDDFT_OK && cudaMemcpy(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = RTTDDFT_ERR_CUDA;
    if (rc == RTTDDFT_OK && (hflag & 8)) rc = RTTDDFT_ERR_TIMEOUT;
    cudaFree(ah);
    cudaFree(al);
    cudaFree(bh);
    cudaFree(bl);
    cudaFree(D);
    cudaFree(flag);
    return rc;
}
