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
#include <cstdlib>
#include <cmath>
#include <string>
#include <vector>

#include "rtd.h"
#include "rttddft.h"

#define TC_BM 128
#define TC_BK 64  // bf16 per K block = 128 bytes, one swizzle row
#define TC_STAGES 4

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// The dynamic shared-memory attribute is global per kernel and shared by every
// context of the process: raise it to `bytes`, never lower it.
static cudaError_t raise_smem(const void* f, int bytes) {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    if (fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

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
// D (TMEM) (+)= A (TMEM, 128 lanes = rows, 16 packed bf16/fp16 K values in 8
// columns) x B (shared-memory descriptor)
__device__ __forceinline__ void umma_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t db, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "r"(tmem_a), "l"(db), "r"(idesc), "r"(accum)
        : "memory");
}
// a warp's 32 lanes x W consecutive 32-bit TMEM columns from W registers per thread
template <int W>
__device__ __forceinline__ void tmem_st(uint32_t taddr, const uint32_t* v) {
    if constexpr (W == 8)
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                     "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                     : "memory");
    else
        asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(v[0]),
                     "r"(v[1]), "r"(v[2]), "r"(v[3])
                     : "memory");
}

// D[split][m][n] (FP32, row-major M x N) = sum over this split's K blocks
// of A^ B^^T; grid (M tiles, K splits, N tiles).
template <int NT>
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
              const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl, int nkb2,
              int kb_per_split, float* __restrict__ D, int M, int N, int* flag) {
    extern __shared__ unsigned char smem_raw[];
    // aligned by offsetting the shared array itself, so that the compiler keeps
    // shared-memory (not generic) addressing for every access through smem
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
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
    if (raise_smem((const void*)k_tc_gemm<NT>, (int)smem) != cudaSuccess)
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

// ============================================================================
// TMA-fed split-BF16 products of the operator apply on the tensor cores:
//   Q[r, n] = sum_G' A[r, G'] C[G', n]          (first factor of Eq. v_MT)
//   Y[G, c] = sum_r conj(A[r, G]) Z[r, c]        (back-projection A^H [hQ | oQ])
// K is cut into blocks of 32 G' (64 reals: 32 Re then 32 Im); the left
// operand of a block is [Re | Im] of 32 entries per row, the right one
// holds, per column n, [Re C | -Im C] (real output rows) and [Im C | Re C]
// (imaginary output rows).  Both operands arrive by TMA (3-D maps over k)
// through one ring of stages; one thread issues the products (hi.hi, hi.lo,
// lo.hi per block); waits are bounded and abort together.
// ============================================================================
#define TCO_GEN 256  // threads of the generating / epilogue warps (8 warps); warp 8 issues, warp 9 copies
#define TCO_THREADS 320
#define TCO_MAXS 4

__device__ bool mbar_wait_ab(uint64_t* b, uint32_t phase, volatile int* ab) {
    const long long t0 = clock64();
    while (!mbar_try_wait(b, phase)) {
        if (*ab) return false;
        if (clock64() - t0 > (1ll << 31)) {
            *ab = 1;
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)tm), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

struct TcOpParams {
    int nk, ns, ma, Dn, kbps, splits, atiles, R, S;
    int nkb_fixed;  // K blocks of every k-point (0: ceil(N_G(k) / 32), or ceil(N_basis(k) / 32) with k_nb)
    int k_nb;       // K runs over the N_basis(k) basis rows
    int rows_ng;    // valid output rows: ma (0), N_G(k) (1) or N_basis(k) (2)
    int fmt;        // operand format: 1 bf16, 0 fp16
    int kofs;  // k-point of blockIdx.z = 0 in the matching-row operand (single-k calls)
    // batched products that are not per k-point (the muffin-tin blocks): a_zmod > 0
    // takes the left operand's slice blockIdx.z % a_zmod and the right operand's
    // blockIdx.z + bz0; the per-k tables are then not read (rows_ng 0, nkb_fixed > 0)
    int a_zmod, bz0;
    int nh;  // > 1: blockIdx.x = tile nh + part, part q takes right-operand rows and output columns q NT ..
    const KDev* kd;
    float* D;  // [nk][splits][R][Dn]
    int* flag;
};

template <int NT>
__global__ void __launch_bounds__(TCO_THREADS, 1)
    k_tc_opfwd(const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
               const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl, TcOpParams p) {
    extern __shared__ unsigned char smem_raw[];
    // aligned by offsetting the shared array itself, so that the compiler keeps
    // shared-memory (not generic) addressing for every access through smem
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    constexpr int A_BYTES = TC_BM * TC_BK * 2;
    constexpr int B_BYTES = NT * TC_BK * 2;
    constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
    // hi.hi and hi.lo as one product of N = 2 NT (B_hi and B_lo are adjacent in
    // shared memory), lo.hi on the first NT columns: two instructions per K step
    constexpr bool MERGE = 2 * NT <= 256;
    constexpr int NACC = MERGE ? 2 * NT : NT;
    constexpr uint32_t NCOLS = NACC <= 32 ? 32 : (NACC <= 64 ? 64 : (NACC <= 128 ? 128 : 256));
    __shared__ __align__(8) uint64_t full[TCO_MAXS], empty[TCO_MAXS], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int S = p.S;
    const int nh = p.nh > 1 ? p.nh : 1;
    const int k = blockIdx.z, tile = blockIdx.x / nh, part = blockIdx.x % nh, split = blockIdx.y;
    const int brow = part * NT;  // first right-operand row and output column of this block
    const bool per_k = p.a_zmod <= 0;
    const int ng = per_k ? p.kd[k].ng : 0;
    const int nbk = per_k ? p.kd[k].nb : 0;
    const int row0 = tile * TC_BM;
    const int nkb = p.nkb_fixed > 0 ? p.nkb_fixed : ((p.k_nb ? nbk : ng) + 31) >> 5;
    const int kb0 = split * p.kbps;
    const int nk = min(nkb, kb0 + p.kbps) - kb0;
    if (nk <= 0) return;  // the reduction skips these slices
    const int rows_valid = p.rows_ng == 2 ? nbk : (p.rows_ng ? ng : p.ma);
    const int za = per_k ? k + p.kofs : k % p.a_zmod, zb = per_k ? k : k + p.bz0;
    if (row0 >= rows_valid) return;  // a row tile past this k-point's rows
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(NCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    volatile int* ab = &abort_flag;
    if (warp == 8) {
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | ((uint32_t)p.fmt << 7) | ((uint32_t)p.fmt << 10) | ((uint32_t)(NT >> 3) << 17) |
                                   ((uint32_t)(TC_BM >> 4) << 24);
            const uint32_t idesc2 = (1u << 4) | ((uint32_t)p.fmt << 7) | ((uint32_t)p.fmt << 10) |
                                    ((uint32_t)((NACC) >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
            for (int j = 0; j < nk; ++j) {
                const int s = j % S;
                if (!mbar_wait_ab(&full[s], (uint32_t)((j / S) & 1), ab)) break;
                tc_fence_after();
                const uint32_t ah = smem_u32(smem + (size_t)s * STAGE), al = ah + A_BYTES;
                const uint32_t bh = ah + 2 * A_BYTES, bl = bh + B_BYTES;
#pragma unroll
                for (int kk = 0; kk < TC_BK / 16; ++kk) {
                    const uint32_t o = kk * 32;
                    if constexpr (MERGE) {
                        umma_bf16(tmem, umma_desc(ah + o), umma_desc(bh + o), idesc2, (j > 0 || kk > 0) ? 1u : 0u);
                        umma_bf16(tmem, umma_desc(al + o), umma_desc(bh + o), idesc, 1u);
                    } else {
                        umma_bf16(tmem, umma_desc(ah + o), umma_desc(bh + o), idesc, (j > 0 || kk > 0) ? 1u : 0u);
                        umma_bf16(tmem, umma_desc(ah + o), umma_desc(bl + o), idesc, 1u);
                        umma_bf16(tmem, umma_desc(al + o), umma_desc(bh + o), idesc, 1u);
                    }
                }
                umma_commit(&empty[s]);
            }
            umma_commit(&done);
            if (*ab) atomicOr(p.flag, 8);
        }
        __syncwarp();
    } else if (warp == 9) {
        // both operands' copies, S blocks ahead of the products: a stage is refilled
        // once the products that read it have completed
        if (lane == 0) {
            int issued = 0;
            for (int j = 0; j < nk; ++j) {
                const int s = j % S, kx = (kb0 + j) * TC_BK;
                if (j >= S && !mbar_wait_ab(&empty[s], (uint32_t)(((j / S) - 1) & 1), ab)) break;
                unsigned char* st = smem + (size_t)s * STAGE;
                mbar_expect_tx(&full[s], STAGE);
                tma_load_3d(st + 2 * A_BYTES, &tmBh, kx, brow, zb, &full[s]);
                tma_load_3d(st + 2 * A_BYTES + B_BYTES, &tmBl, kx, brow, zb, &full[s]);
                tma_load_3d(st, &tmAh, kx, row0, za, &full[s]);
                tma_load_3d(st + A_BYTES, &tmAl, kx, row0, za, &full[s]);
                issued = j + 1;
            }
            if (*ab) {
                // the copies in flight land before the block's shared memory goes away
                for (int j = max(0, issued - S); j < issued; ++j) mbar_wait(&full[j % S], (uint32_t)((j / S) & 1));
            }
        }
        __syncwarp();
    }
    __syncthreads();
    const bool okd = mbar_wait(&done, 0);
    tc_fence_after();
    if (warp < 8 && okd && !*ab) {
        const int q = warp & 3, half = warp >> 2;
        const int lrow = row0 + q * 32 + lane;
        float* drow = p.D + (((size_t)k * p.splits + split) * p.R + lrow) * p.Dn + brow;
#pragma unroll 1
        for (int c = half * (NT / 2); c < (half + 1) * (NT / 2); c += 8) {
            uint32_t v[8];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                : "r"(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c));
            uint32_t v2[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
            if constexpr (MERGE)
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                    : "=r"(v2[0]), "=r"(v2[1]), "=r"(v2[2]), "=r"(v2[3]), "=r"(v2[4]), "=r"(v2[5]), "=r"(v2[6]),
                      "=r"(v2[7])
                    : "r"(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(NT + c)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (lrow < rows_valid) {
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (brow + c + u < p.Dn) drow[c + u] = __uint_as_float(v[u]) + __uint_as_float(v2[u]);
            }
        }
    } else if (tid == 0 && !okd) {
        atomicOr(p.flag, 8);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 8)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS) : "memory");
}

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t*>(&v); }

// ============================================================================
// The interstitial rows alone (T[G, n] = sum_G' V~_{G-G'} C[G', n]) with two
// rings: SA stages of the generated left operand (256 threads write the
// hi/lo tiles from the pre-split table window by byte permutes) and SB
// deeper stages of the small TMA-fed right operand, so that the copy
// latency of the right operand stays hidden behind several K blocks.
// ============================================================================
#define TCT_MAXSA 4
#define TCT_MAXSB 16
struct TcToepParams {
    int nk, Dn, kbps, splits, ttiles, wcap, vt_center, SA, SB;
    int fmt;    // operand format: 1 bf16, 0 fp16
    int brow0;  // first row of the right operand's tile (column tiles of wide products)
    const KDev* kd;
    const uint2* tab;  // pre-split table
    float* D;          // [nk][splits][ttiles * 128][Dn]
    int* flag;
};

template <int NT, bool GW, int GEN, bool TA>
__global__ void __launch_bounds__(GEN + 64, 1)
    k_tc_toep(const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl, TcToepParams p) {
    // TA: the generated left operand goes to tensor memory (tcgen05.st, 64 columns a
    // stage from column 256: hi Re | hi Im | lo Re | lo Im, 16 columns each) and the
    // products read it there, instead of a swizzled shared-memory tile: no shared-
    // memory traffic and no proxy fence for the left operand.
    // GW: gather the table from global memory (L1/L2) instead of a shared window.
    // GEN: generating threads (256 or 512: 2 or 4 per output row, each writing 16 or
    // 8 G' of a K block, with the table loads of 1 or 3 blocks ahead in flight).
    static_assert(GEN == 256 || GEN == 512, "two or four generating threads per row");
    constexpr int PER = 32 * TC_BM / GEN;  // G' per thread and K block
    constexpr int MW = GEN / 32;           // the issuing warp; warp MW + 1 copies the right operand
    extern __shared__ unsigned char smem_raw[];
    // aligned by offsetting the shared array itself, so that the compiler keeps
    // shared-memory (not generic) addressing for every access through smem
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    constexpr int A_BYTES = TC_BM * TC_BK * 2;
    constexpr int B_BYTES = NT * TC_BK * 2;
    // hi.hi and hi.lo as one product of N = 2 NT (B_hi and B_lo are adjacent in
    // shared memory), lo.hi on the first NT columns: two instructions per K step
    constexpr bool MERGE = 2 * NT <= 256;
    constexpr int NACC = MERGE ? 2 * NT : NT;
    constexpr uint32_t NCOLS_ACC = NACC <= 32 ? 32 : (NACC <= 64 ? 64 : (NACC <= 128 ? 128 : 256));
    constexpr uint32_t NCOLS = TA ? 512 : NCOLS_ACC;
    constexpr uint32_t ACOL0 = 256;  // TA: first column of the left-operand stages
    static_assert(!TA || TCT_MAXSA * 64 + ACOL0 <= 512, "left-operand stages beyond tensor memory");
    __shared__ __align__(8) uint64_t fullA[TCT_MAXSA], emptyA[TCT_MAXSA], fullB[TCT_MAXSB], emptyB[TCT_MAXSB], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int SA = p.SA, SB = p.SB;
    const int k = blockIdx.z, tile = blockIdx.x, split = blockIdx.y;
    const KDev& K = p.kd[k];
    const int ng = K.ng;
    const int row0 = tile * TC_BM;
    const int nkb = (ng + 31) >> 5;
    const int kb0 = split * p.kbps;
    const int nk = min(nkb, kb0 + p.kbps) - kb0;
    if (nk <= 0 || row0 >= ng) return;  // the reduction skips these pairs
    unsigned char* ringA = smem;
    unsigned char* ringB = smem + (TA ? (size_t)0 : (size_t)SA * 2 * A_BYTES);
    int* gl_s = (int*)(ringB + (size_t)SB * 2 * B_BYTES);
    uint2* win = (uint2*)(gl_s + p.kbps * 32);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < SA; ++s) {
            mbar_init(&fullA[s], MW);
            mbar_init(&emptyA[s], 1);
        }
        for (int s = 0; s < SB; ++s) {
            mbar_init(&fullB[s], 1);
            mbar_init(&emptyB[s], 1);
        }
        mbar_init(&done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == MW) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(NCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    const int gp_lo = kb0 * 32, gp_hi = min(ng, (kb0 + nk) * 32);
    int wlo = 0;
    if (tid < GEN) {
        const int* __restrict__ glin = K.glin;
        const int g1 = min(row0 + TC_BM, ng) - 1;
        wlo = glin[row0] - glin[gp_hi - 1] + p.vt_center;
        if constexpr (!GW) {
            const int wn = glin[g1] - glin[gp_lo] + p.vt_center - wlo + 1;
            if (wn > p.wcap) {
                // the host sizes the slices so that this cannot happen
                abort_flag = 1;
                if (tid == 0) atomicOr(p.flag, 8);
            } else {
                for (int e = tid; e < wn; e += GEN) win[e] = p.tab[wlo + e];
            }
        }
        for (int i = tid; i < gp_hi - gp_lo; i += GEN) gl_s[i] = glin[gp_lo + i];
    }
    const uint2* __restrict__ gtab = p.tab + wlo;  // GW: the same offsets into the table
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    volatile int* ab = &abort_flag;
    if (warp == MW) {
        if (lane == 0 && *ab) {
            umma_commit(&done);
        } else if (lane == 0) {
            const uint32_t idesc = (1u << 4) | ((uint32_t)p.fmt << 7) | ((uint32_t)p.fmt << 10) | ((uint32_t)(NT >> 3) << 17) |
                                   ((uint32_t)(TC_BM >> 4) << 24);
            const uint32_t idesc2 = (1u << 4) | ((uint32_t)p.fmt << 7) | ((uint32_t)p.fmt << 10) |
                                    ((uint32_t)((NACC) >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
            for (int j = 0; j < nk; ++j) {
                const int sa = j % SA, sb = j % SB;
                if (!mbar_wait_ab(&fullB[sb], (uint32_t)((j / SB) & 1), ab)) break;
                if (!mbar_wait_ab(&fullA[sa], (uint32_t)((j / SA) & 1), ab)) break;
                tc_fence_after();
                const uint32_t bh = smem_u32(ringB + (size_t)sb * 2 * B_BYTES), bl = bh + B_BYTES;
                if constexpr (TA) {
                    const uint32_t th = tmem + ACOL0 + 64u * (uint32_t)sa, tl = th + 32u;
#pragma unroll
                    for (int kk = 0; kk < TC_BK / 16; ++kk) {
                        const uint32_t o = kk * 32, c = kk * 8;
                        if constexpr (MERGE) {
                            umma_ts(tmem, th + c, umma_desc(bh + o), idesc2, (j > 0 || kk > 0) ? 1u : 0u);
                            umma_ts(tmem, tl + c, umma_desc(bh + o), idesc, 1u);
                        } else {
                            umma_ts(tmem, th + c, umma_desc(bh + o), idesc, (j > 0 || kk > 0) ? 1u : 0u);
                            umma_ts(tmem, th + c, umma_desc(bl + o), idesc, 1u);
                            umma_ts(tmem, tl + c, umma_desc(bh + o), idesc, 1u);
                        }
                    }
                } else {
                    const uint32_t ah = smem_u32(ringA + (size_t)sa * 2 * A_BYTES), al = ah + A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < TC_BK / 16; ++kk) {
                        const uint32_t o = kk * 32;
                        if constexpr (MERGE) {
                            umma_bf16(tmem, umma_desc(ah + o), umma_desc(bh + o), idesc2, (j > 0 || kk > 0) ? 1u : 0u);
                            umma_bf16(tmem, umma_desc(al + o), umma_desc(bh + o), idesc, 1u);
                        } else {
                            umma_bf16(tmem, umma_desc(ah + o), umma_desc(bh + o), idesc, (j > 0 || kk > 0) ? 1u : 0u);
                            umma_bf16(tmem, umma_desc(ah + o), umma_desc(bl + o), idesc, 1u);
                            umma_bf16(tmem, umma_desc(al + o), umma_desc(bh + o), idesc, 1u);
                        }
                    }
                }
                umma_commit(&emptyA[sa]);
                umma_commit(&emptyB[sb]);
            }
            umma_commit(&done);
            if (*ab) atomicOr(p.flag, 8);
        }
        __syncwarp();
    } else if (warp == MW + 1) {
        // the right operand's copies, SB blocks ahead of the products: a stage is
        // refilled once the products that read it have completed
        if (lane == 0 && !*ab) {
            int issued = 0;
            for (int j = 0; j < nk; ++j) {
                const int s = j % SB;
                if (j >= SB && !mbar_wait_ab(&emptyB[s], (uint32_t)(((j / SB) - 1) & 1), ab)) break;
                unsigned char* st = ringB + (size_t)s * 2 * B_BYTES;
                const int kx = (kb0 + j) * TC_BK;
                mbar_expect_tx(&fullB[s], 2 * B_BYTES);
                tma_load_3d(st, &tmBh, kx, p.brow0, k, &fullB[s]);
                tma_load_3d(st + B_BYTES, &tmBl, kx, p.brow0, k, &fullB[s]);
                issued = j + 1;
            }
            if (*ab) {
                // the copies in flight land before the block's shared memory goes away
                for (int j = max(0, issued - SB); j < issued; ++j) mbar_wait(&fullB[j % SB], (uint32_t)((j / SB) & 1));
            }
        }
        __syncwarp();
    } else if (!*ab) {
        // generators: thread (r, h) writes row r, G' PER h .. PER h + PER - 1 of every
        // K block.  The table entries of block j + 1 are fetched before block j is
        // written, so that their latency (L1/L2 in the gather form) overlaps the
        // permutes and stores.
        const int r = tid & (TC_BM - 1), h = tid >> 7;
        const int g = row0 + r;
        const bool valid = g < ng;
        const int lb = (valid ? K.glin[g] : 0) + p.vt_center - wlo;
        const uint32_t sw = (uint32_t)(r & 7);
        auto fetch = [&](int j, uint2* u) {
            const int gq = (kb0 + j) * 32 + PER * h;
            if (valid && gq + PER <= gp_hi) {
                const int4* g4 = (const int4*)(gl_s + (gq - gp_lo));
#pragma unroll
                for (int q = 0; q < PER / 4; ++q) {
                    const int4 t = g4[q];
                    if constexpr (GW) {
                        u[4 * q + 0] = __ldg(gtab + (lb - t.x));
                        u[4 * q + 1] = __ldg(gtab + (lb - t.y));
                        u[4 * q + 2] = __ldg(gtab + (lb - t.z));
                        u[4 * q + 3] = __ldg(gtab + (lb - t.w));
                    } else {
                        u[4 * q + 0] = win[lb - t.x];
                        u[4 * q + 1] = win[lb - t.y];
                        u[4 * q + 2] = win[lb - t.z];
                        u[4 * q + 3] = win[lb - t.w];
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < PER; ++i) {
                    const int gp = gq + i;
                    if (valid && gp < gp_hi) {
                        const int x = lb - gl_s[gp - gp_lo];
                        u[i] = GW ? __ldg(gtab + x) : win[x];
                    } else {
                        u[i] = make_uint2(0u, 0u);
                    }
                }
            }
        };
        auto store = [&](int j, const uint2* u) -> bool {
            const int sa = j % SA;
            // warp-uniform: the stores below are whole-warp instructions
            const bool okw = (j < SA) || mbar_wait_ab(&emptyA[sa], (uint32_t)(((j / SA) - 1) & 1), ab);
            if (!__all_sync(0xffffffffu, okw)) return false;
            if constexpr (TA) {
                // the row's words in the warp's lane quadrant: word q of a part holds
                // G' PER h + 2q (low half) and + 2q + 1 (high half)
                tc_fence_after();
                constexpr int W = PER / 2;
                uint32_t rh[W], ih[W], rl[W], il[W];
#pragma unroll
                for (int q = 0; q < W; ++q) {
                    rh[q] = __byte_perm(u[2 * q].x, u[2 * q + 1].x, 0x5410);
                    ih[q] = __byte_perm(u[2 * q].y, u[2 * q + 1].y, 0x5410);
                    rl[q] = __byte_perm(u[2 * q].x, u[2 * q + 1].x, 0x7632);
                    il[q] = __byte_perm(u[2 * q].y, u[2 * q + 1].y, 0x7632);
                }
                const uint32_t t0 = tmem + ((uint32_t)((warp & 3) * 32) << 16) + ACOL0 + 64u * (uint32_t)sa +
                                    (uint32_t)(W * h);
                tmem_st<W>(t0, rh);
                tmem_st<W>(t0 + 16, ih);
                tmem_st<W>(t0 + 32, rl);
                tmem_st<W>(t0 + 48, il);
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&fullA[sa]);
                return true;
            }
            unsigned char* rowp = ringA + (size_t)sa * 2 * A_BYTES + r * 128;
#pragma unroll
            for (int q = 0; q < PER / 8; ++q) {
                const uint2* w = u + 8 * q;
                const uint32_t cre = (uint32_t)((PER / 8) * h + q), cim = cre + 4;
                uint4* p0 = (uint4*)(rowp + ((cre ^ sw) << 4));
                uint4* p1 = (uint4*)(rowp + ((cim ^ sw) << 4));
                *p0 = make_uint4(__byte_perm(w[0].x, w[1].x, 0x5410), __byte_perm(w[2].x, w[3].x, 0x5410),
                                 __byte_perm(w[4].x, w[5].x, 0x5410), __byte_perm(w[6].x, w[7].x, 0x5410));
                *p1 = make_uint4(__byte_perm(w[0].y, w[1].y, 0x5410), __byte_perm(w[2].y, w[3].y, 0x5410),
                                 __byte_perm(w[4].y, w[5].y, 0x5410), __byte_perm(w[6].y, w[7].y, 0x5410));
                *(uint4*)((unsigned char*)p0 + A_BYTES) =
                    make_uint4(__byte_perm(w[0].x, w[1].x, 0x7632), __byte_perm(w[2].x, w[3].x, 0x7632),
                               __byte_perm(w[4].x, w[5].x, 0x7632), __byte_perm(w[6].x, w[7].x, 0x7632));
                *(uint4*)((unsigned char*)p1 + A_BYTES) =
                    make_uint4(__byte_perm(w[0].y, w[1].y, 0x7632), __byte_perm(w[2].y, w[3].y, 0x7632),
                               __byte_perm(w[4].y, w[5].y, 0x7632), __byte_perm(w[6].y, w[7].y, 0x7632));
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&fullA[sa]);
            return true;
        };
        // NB register sets in turn: the loads of the next NB - 1 blocks stay in
        // flight while a block is written (2 sets with 16 G' per thread, 4 with 8)
        constexpr int NB = (GEN == 512) ? 4 : 2;
        uint2 ub[NB][PER];
#pragma unroll
        for (int q = 0; q < NB - 1; ++q)
            if (q < nk) fetch(q, ub[q]);
        bool going = true;
        for (int j0 = 0; j0 < nk && going; j0 += NB) {
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const int j = j0 + q;
                if (j >= nk) break;
                if (j + NB - 1 < nk) fetch(j + NB - 1, ub[(q + NB - 1) % NB]);
                if (!store(j, ub[q])) {
                    going = false;
                    break;
                }
            }
        }
    }
    __syncthreads();
    const bool okd = mbar_wait(&done, 0);
    tc_fence_after();
    if (warp < MW && okd && !*ab) {
        // warp w reads the TMEM lanes of its quadrant w % 4 (32 rows), every
        // (MW / 4)-th group of 8 columns
        const int q = warp & 3, part = warp >> 2;
        const int lrow = row0 + q * 32 + lane;
        float* drow = p.D + (((size_t)k * p.splits + split) * ((size_t)p.ttiles * TC_BM) + lrow) * p.Dn;
#pragma unroll 1
        for (int c = part * 8; c < NT; c += 2 * MW) {
            uint32_t v[8];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                : "r"(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c));
            uint32_t v2[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
            if constexpr (MERGE)
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                    : "=r"(v2[0]), "=r"(v2[1]), "=r"(v2[2]), "=r"(v2[3]), "=r"(v2[4]), "=r"(v2[5]), "=r"(v2[6]),
                      "=r"(v2[7])
                    : "r"(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(NT + c)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (lrow < ng) {
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (c + u < p.Dn) drow[c + u] = __uint_as_float(v[u]) + __uint_as_float(v2[u]);
            }
        }
    } else if (tid == 0 && !okd) {
        atomicOr(p.flag, 8);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == MW)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS) : "memory");
}

// the pre-split table of the tensor-core form (set-up)
__global__ void k_tc_split_table(const zd* __restrict__ t, uint2* __restrict__ out, int n, int fmt, double scale,
                                 int* flag) {
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    bool o1, o2;
    out[i] = make_uint2(split16_bits(t[i].x, fmt, scale, o1), split16_bits(t[i].y, fmt, scale, o2));
    if (!(o1 && o2)) atomicOr(flag, 32);
}

// store the scaled split of v at hi[i], lo[i]; flag bit 5 when out of the fp16 range
__device__ __forceinline__ void put16(double v, int fmt, double scale, unsigned short* hi, unsigned short* lo,
                                      size_t i, int* flag) {
    unsigned short h, l;
    if (!split16(v, fmt, scale, h, l)) atomicOr(flag, 32);
    hi[i] = h;
    lo[i] = l;
}

// Right operand of a step: B^[k][row][K-block layout] from C_G (FP64, the
// first ng rows of K.C), scaled by sc.  Rows 2 ns .. and G' >= ng stay zero.
__global__ void k_tc_pack_c(const KDev* __restrict__ kd, int ns, int Kp, int Rp, unsigned short* __restrict__ bh,
                            unsigned short* __restrict__ bl, int fmt, double sc, int* flag) {
    const int k = blockIdx.z;
    const KDev& K = kd[k];
    const int ng = K.ng;
    const int e = blockIdx.x * 256 + threadIdx.x;  // (n, G') pair
    if (e >= ns * ng) return;
    const int n = e / ng, gp = e % ng;
    const zd c = K.C[gp + (size_t)n * K.nb];
    const int kb = gp >> 5, o = gp & 31;
    const size_t re_row = ((size_t)k * Rp + n) * Kp + (size_t)kb * 64;
    const size_t im_row = ((size_t)k * Rp + ns + n) * Kp + (size_t)kb * 64;
    put16(c.x, fmt, sc, bh, bl, re_row + o, flag);
    put16(c.x, fmt, sc, bh, bl, im_row + 32 + o, flag);
    put16(c.y, fmt, sc, bh, bl, im_row + o, flag);
    put16(-c.y, fmt, sc, bh, bl, re_row + 32 + o, flag);
}

// Left operand of the matching rows (set-up): A^[k][r][K-block layout] with
// A[r, G'] = conj(AT[G' + r ng]), scaled by sa.
__global__ void k_tc_pack_at(const zd* __restrict__ at, int ng, int ma, int Kp, int Mp, int k,
                             unsigned short* __restrict__ ah, unsigned short* __restrict__ al, int fmt, double sa,
                             int* flag) {
    const size_t e = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (e >= (size_t)ma * ng) return;
    const int gp = (int)(e % ng), r = (int)(e / ng);
    const zd a = at[gp + (size_t)r * ng];
    const size_t row = ((size_t)k * Mp + r) * Kp + (size_t)(gp >> 5) * 64 + (gp & 31);
    put16(a.x, fmt, sa, ah, al, row, flag);
    put16(-a.y, fmt, sa, ah, al, row + 32, flag);
}

// Left operand of the back-projection (set-up): A^[k][G][K-block layout over
// the matching rows r], the entry A^H[G, r] = AT[G + r ng], scaled by sa.
__global__ void k_tc_pack_atb(const zd* __restrict__ at, int ng, int ma, int Kp, int Mp, int k,
                              unsigned short* __restrict__ ah, unsigned short* __restrict__ al, int fmt, double sa,
                              int* flag) {
    const size_t e = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (e >= (size_t)ma * ng) return;
    const int g = (int)(e % ng), r = (int)(e / ng);
    const zd a = at[g + (size_t)r * ng];
    const size_t row = ((size_t)k * Mp + g) * Kp + (size_t)(r >> 5) * 64 + (r & 31);
    put16(a.x, fmt, sa, ah, al, row, flag);
    put16(a.y, fmt, sa, ah, al, row + 32, flag);
}

// Right operand of the back-projection (per step) from Z = [hQ | oQ]
// (ma x 2 ns, FP64), scaled by sz: rows c < 2 ns hold [Re Z | -Im Z], rows
// 2 ns + c hold [Im Z | Re Z] over the matching rows.
__global__ void k_tc_pack_z(const KDev* __restrict__ kd, int ns, int ma, int Kp, int Rp,
                            unsigned short* __restrict__ bh, unsigned short* __restrict__ bl, int fmt, double sz,
                            int* flag) {
    const int k = blockIdx.z;
    const KDev& K = kd[k];
    const int nc = 2 * ns;
    const int e = blockIdx.x * 256 + threadIdx.x;  // (c, r) pair
    if (e >= nc * ma) return;
    const int c = e / ma, r = e % ma;
    const zd z = K.Z[r + (size_t)c * ma];
    const int kb = r >> 5, o = r & 31;
    const size_t re_row = ((size_t)k * Rp + c) * Kp + (size_t)kb * 64;
    const size_t im_row = ((size_t)k * Rp + nc + c) * Kp + (size_t)kb * 64;
    put16(z.x, fmt, sz, bh, bl, re_row + o, flag);
    put16(z.x, fmt, sz, bh, bl, im_row + 32 + o, flag);
    put16(z.y, fmt, sz, bh, bl, im_row + o, flag);
    put16(-z.y, fmt, sz, bh, bl, re_row + 32 + o, flag);
}

// Sum of the K slices (two-sum pairs, FP64 results): interstitial rows into K.th (ng x ns),
// matching rows into K.Q (ma x ns).
struct TcRedParams {
    int ns, ma, Dn, kbps_t, splits_t, kbps_a, splits_a, Rt, Ra;
    int part;  // 0: interstitial and matching rows, 1: interstitial only, 2: matching only, 3: back-projection
    int Dnb, kbps_b, splits_b, nkb_b, Rb;
    int maxng;                   // largest N_G (the row tiles of the interstitial part)
    double inv_t, inv_a, inv_b;  // undo the operand scales of the split-FP16 form
    const KDev* kd;
    const float* Dt;
    const float* Da;
    const float* Db;
};
// Sum of FP32 values kept as an unevaluated pair s + e (Knuth's two-sum on each
// addition, the rounding errors collected in e): FP32 arithmetic throughout, so
// a sum of a few slices costs no FP64 instructions until the pair is widened
// once; it carries about 48 significant bits, more than the slices' own.
struct Sum2f {
    float s = 0.f, e = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x, bp = t - s;
        e += (s - (t - bp)) + (x - bp);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)e; }
};
// A tile of TC_RT output rows of one product: the FP32 slice partials
// D[s][row][Dn] (real columns c < nc: Re, nc + c: Im) summed over the nsp
// slices in slice order (two-sum pairs, widened to FP64 once), staged in
// shared memory so that the loads run along the rows of D and the stores
// along the columns of the column-major output out[row + c ld].
#define TC_RT 16
__device__ void tc_red_tile(const float* __restrict__ D, size_t sstride, int nsp, int Dn, int nc, int row0,
                            int nrow, double scale, zd* __restrict__ out, size_t ld, double (*tile)[257]) {
    const int n2 = 2 * nc;
    if ((n2 & 3) == 0 && (Dn & 3) == 0 && (sstride & 3) == 0 && ((uintptr_t)D & 15) == 0) {
        // four adjacent columns per thread (16-byte loads), the same slice order
        const int q4 = n2 >> 2;
        for (int e = threadIdx.x; e < TC_RT * q4; e += blockDim.x) {
            const int r = e / q4, c = (e % q4) * 4, row = row0 + r;
            Sum2f v0, v1, v2, v3;
            if (row < nrow) {
                const float* d = D + (size_t)row * Dn + c;
                for (int s0 = 0; s0 < nsp; s0 += 4) {
                    float4 a[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        a[u] = (s0 + u < nsp) ? __ldcs((const float4*)(d + (size_t)(s0 + u) * sstride))
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        v0.add(a[u].x);
                        v1.add(a[u].y);
                        v2.add(a[u].z);
                        v3.add(a[u].w);
                    }
                }
            }
            tile[r][c] = v0.value();
            tile[r][c + 1] = v1.value();
            tile[r][c + 2] = v2.value();
            tile[r][c + 3] = v3.value();
        }
    } else {
        for (int e = threadIdx.x; e < TC_RT * n2; e += blockDim.x) {
            const int r = e / n2, c = e % n2, row = row0 + r;
            Sum2f v;
            if (row < nrow) {
                const float* d = D + (size_t)row * Dn + c;
                for (int s0 = 0; s0 < nsp; s0 += 4) {
                    float a[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) a[u] = (s0 + u < nsp) ? d[(size_t)(s0 + u) * sstride] : 0.f;
#pragma unroll
                    for (int u = 0; u < 4; ++u) v.add(a[u]);
                }
            }
            tile[r][c] = v.value();
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TC_RT * nc; e += blockDim.x) {
        const int r = e % TC_RT, c = e / TC_RT, row = row0 + r;
        if (row < nrow) out[row + (size_t)c * ld] = zmk(tile[r][c] * scale, tile[r][nc + c] * scale);
    }
}

// Split-K sums of the operator's tensor-core products: the interstitial rows
// into K.th and the matching rows into K.Q (part 0, or 1 / 2 for one of
// them), the back-projection into K.tb (part 3).  Blocks: row tiles of the
// interstitial rows (over the largest N_G), then of the matching rows.
__global__ void __launch_bounds__(256) k_tc_opred(TcRedParams p) {
    __shared__ double tile[TC_RT][257];
    const int k = blockIdx.z;
    const KDev& K = p.kd[k];
    const int ng = K.ng, ns = p.ns;
    const int nkb = (ng + 31) >> 5;
    if (p.part == 3) {
        const int nsp = min(p.splits_b, (p.nkb_b + p.kbps_b - 1) / p.kbps_b);
        const int row0 = blockIdx.x * TC_RT;
        if (row0 >= ng) return;
        tc_red_tile(p.Db + (size_t)k * p.splits_b * p.Rb * p.Dnb, (size_t)p.Rb * p.Dnb, nsp, p.Dnb, 2 * ns, row0, ng,
                    p.inv_b, K.tb, ng, tile);
        return;
    }
    const int tiles_t = (p.part == 2) ? 0 : (p.maxng + TC_RT - 1) / TC_RT;
    if ((int)blockIdx.x < tiles_t) {
        const int row0 = blockIdx.x * TC_RT;
        if (row0 >= ng) return;
        const int nsp = min(p.splits_t, (nkb + p.kbps_t - 1) / p.kbps_t);
        tc_red_tile(p.Dt + (size_t)k * p.splits_t * p.Rt * p.Dn, (size_t)p.Rt * p.Dn, nsp, p.Dn, ns, row0, ng, p.inv_t,
                    K.th, ng, tile);
    } else if (p.part != 1) {
        const int row0 = (blockIdx.x - tiles_t) * TC_RT;
        if (row0 >= p.ma) return;
        const int nsp = min(p.splits_a, (nkb + p.kbps_a - 1) / p.kbps_a);
        tc_red_tile(p.Da + (size_t)k * p.splits_a * p.Ra * p.Dn, (size_t)p.Ra * p.Dn, nsp, p.Dn, ns, row0, p.ma,
                    p.inv_a, K.Q, p.ma, tile);
    }
}
static dim3 tc_red_grid(int part, int maxng, int ma, int nk) {
    const int tt = (maxng + TC_RT - 1) / TC_RT, ta = (ma + TC_RT - 1) / TC_RT;
    if (part == 3 || part == 1) return dim3(tt, 1, nk);
    if (part == 2) return dim3(ta, 1, nk);
    return dim3(tt + ta, 1, nk);
}

// ------------------------------------------------------------ operator plan
struct TcPlan {
    int nk = 0, ns = 0, ma = 0, Dn = 0, NT = 0, ttiles = 0, atiles = 0, Kp = 0, Mp = 0, Rp = 0;
    int maxng = 0, vt_center = 0;
    // interstitial rows
    int SA = 0, SB = 0, kbps_t = 0, splits_t = 0, wcap = 0, gen_t = 256, ta_t = 0;
    size_t smem_t = 0;
    // matching rows
    int S_a = 0, kbps_a = 0, splits_a = 0;
    size_t smem_a = 0;
    CUtensorMap tbh, tbl, tah, tal;
    unsigned short *bh = nullptr, *bl = nullptr, *ah = nullptr, *al = nullptr;  // 16-bit operand splits
    float *Dt = nullptr, *Da = nullptr;
    int fmt = 1;                                    // 1 bf16, 0 fp16
    double sA = 1.0, sT = 1.0, sC = 1.0, sZ = 1.0;  // operand scales (powers of two)
    uint2* tabs = nullptr;  // the pre-split static table
    int* tflag = nullptr;   // error flag of the tuning launches
    float ms_t = 0.f, ms_a = 0.f;  // tuned launch times
    int ncand = 0;
    // potential-change rebuild T = dV~ * CC_G (Eq. v_interstitial), N_aux columns in
    // tiles of 128 complex columns, split-BF16, table gathered through L2
    int dv_ready = 0, naux = 0, dv_tiles = 0, dv_kbps = 0, dv_splits = 0;
    double dv_sc = 1.0, dv_st = 1.0;  // fp16 form: scales of the packed CC_G and of the split dV~ table
    size_t dv_smem = 0;
    CUtensorMap tch, tcl;
    unsigned short *cch = nullptr, *ccl = nullptr;
    uint2* dvtabs = nullptr;
    float* Dd = nullptr;
    // back-projection Y_G = A^H [hQ | oQ]: rows G, K over the matching rows
    int NTb = 0, Dnb = 0, nkb_b = 0, Kpb = 0, Rpb = 0, S_b = 0, kbps_b = 0, splits_b = 0, nh_b = 1;
    size_t smem_b = 0;
    float ms_b = 0.f;
    CUtensorMap tzh, tzl, tabh, tabl;
    CUtensorMap tzh2, tzl2;  // the right operand in boxes of 128 rows (column parts)
    unsigned short *zh = nullptr, *zl = nullptr, *abh = nullptr, *abl = nullptr;
    float* Db = nullptr;
};

static const int TCO_NTS[] = {16, 32, 48, 64, 96, 128, 160, 192, 224, 256};

// largest table window over every (k, row tile, K slice of kbps blocks)
static int tco_max_window(int nk, const int* ng, const int* const* glin, int kbps) {
    int w = 0;
    for (int k = 0; k < nk; ++k) {
        const int n = ng[k], nkb = (n + 31) / 32;
        const int* gl = glin[k];
        for (int t0 = 0; t0 < n; t0 += TC_BM) {
            const int g1 = std::min(t0 + TC_BM, n) - 1;
            for (int kb0 = 0; kb0 < nkb; kb0 += kbps) {
                const int lo = kb0 * 32, hi = std::min(n, (kb0 + kbps) * 32);
                w = std::max(w, gl[g1] - gl[lo] - (gl[t0] - gl[hi - 1]) + 1);
            }
        }
    }
    return w;
}

static int tc_tmap3(CUtensorMap* tm, const void* base, uint64_t inner, uint64_t rows, uint64_t depth,
                    uint32_t box_rows) {
    encode_fn_t enc = get_encode();
    if (!enc) return -1;
    if ((uintptr_t)base & 15) return -2;
    cuuint64_t dims[3] = {inner, rows, depth};
    cuuint64_t strides[2] = {inner * 2, inner * rows * 2};
    cuuint32_t box[3] = {TC_BK, box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -3;
}

template <int NT>
static cudaError_t tco_set_smem(int bytes_opfwd, int bytes_toep) {
    cudaError_t e = raise_smem((const void*)k_tc_opfwd<NT>, bytes_opfwd);
    if (e != cudaSuccess) return e;
    const void* fs[] = {(const void*)k_tc_toep<NT, false, 256, false>, (const void*)k_tc_toep<NT, true, 256, false>,
                        (const void*)k_tc_toep<NT, true, 512, false>, (const void*)k_tc_toep<NT, true, 256, true>,
                        (const void*)k_tc_toep<NT, true, 512, true>};
    for (const void* f : fs) {
        e = raise_smem(f, bytes_toep);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void tc_plan_destroy(TcPlan* tp) {
    if (!tp) return;
    cudaFree(tp->bh);
    cudaFree(tp->bl);
    cudaFree(tp->ah);
    cudaFree(tp->al);
    cudaFree(tp->Dt);
    cudaFree(tp->Da);
    cudaFree(tp->tabs);
    cudaFree(tp->tflag);
    cudaFree(tp->cch);
    cudaFree(tp->ccl);
    cudaFree(tp->dvtabs);
    cudaFree(tp->Dd);
    cudaFree(tp->zh);
    cudaFree(tp->zl);
    cudaFree(tp->abh);
    cudaFree(tp->abl);
    cudaFree(tp->Db);
    delete tp;
}

// waves x (K blocks per slice + 2 for fill and drain), a small charge per slice
static int tco_best_splits(int tiles, int nk, int nkb, int nsm, int per_sm) {
    int best = 1;
    double bcost = 1e30;
    for (int sp = 1; sp <= nkb; ++sp) {
        const int kb = (nkb + sp - 1) / sp;
        const double waves = std::ceil((double)tiles * nk * sp / ((double)nsm * per_sm));
        const double cost = waves * (kb + 2) + 0.02 * sp;
        if (cost < bcost) {
            bcost = cost;
            best = sp;
        }
    }
    return best;
}

// one launch of the interstitial kernel in the variant (window or gather, generating
// threads, left operand in shared or tensor memory)
template <int NT>
static void toep_variant(int wn, int gen, int ta, dim3 g, size_t smem, cudaStream_t s, const CUtensorMap& bh,
                         const CUtensorMap& bl, const TcToepParams& p) {
    // generating warps + the issuing warp + the copy warp
    if (wn > 0) k_tc_toep<NT, false, 256, false><<<g, 256 + 64, smem, s>>>(bh, bl, p);
    else if (gen == 512 && ta) k_tc_toep<NT, true, 512, true><<<g, 512 + 64, smem, s>>>(bh, bl, p);
    else if (gen == 512) k_tc_toep<NT, true, 512, false><<<g, 512 + 64, smem, s>>>(bh, bl, p);
    else if (ta) k_tc_toep<NT, true, 256, true><<<g, 256 + 64, smem, s>>>(bh, bl, p);
    else k_tc_toep<NT, true, 256, false><<<g, 256 + 64, smem, s>>>(bh, bl, p);
}

struct TcToepCand {
    int kbps, splits, SA, SB, wn;  // wn = 0: table gathered from global memory
    int gen;                       // generating threads (512 only with the gathered table)
    int ta;                        // left operand in tensor memory (gathered table only)
    size_t smem;
    float ms;
};
struct TcRowsCand {
    int kbps, splits, S;
    size_t smem;
    float ms;
    int nh;  // back-projection: output column parts of 128 (1: one part of NTb)
};

template <int NT>
static void tco_launch_toep(const TcPlan* tp, const TcToepCand& c, const KDev* kd, int nk, cudaStream_t s) {
    TcToepParams p{};
    p.nk = nk;
    p.Dn = tp->Dn;
    p.kbps = c.kbps;
    p.splits = c.splits;
    p.ttiles = tp->ttiles;
    p.wcap = c.wn;
    p.vt_center = tp->vt_center;
    p.SA = c.SA;
    p.SB = c.SB;
    p.fmt = tp->fmt;
    p.kd = kd;
    p.tab = tp->tabs;
    p.D = tp->Dt;
    p.flag = tp->tflag;
    toep_variant<NT>(c.wn, c.gen, c.ta, dim3(tp->ttiles, c.splits, nk), c.smem, s, tp->tbh, tp->tbl, p);
    // with the sum of its slices, so that many slices pay for their reduction
    TcRedParams r{};
    r.ns = tp->ns;
    r.ma = tp->ma;
    r.Dn = tp->Dn;
    r.kbps_t = c.kbps;
    r.splits_t = c.splits;
    r.Rt = tp->ttiles * TC_BM;
    r.part = 1;
    r.inv_t = 1.0 / (tp->sT * tp->sC);
    r.kd = kd;
    r.Dt = tp->Dt;
    r.maxng = tp->maxng;
    k_tc_opred<<<tc_red_grid(r.part, tp->maxng, tp->ma, nk), 256, 0, s>>>(r);
}
template <int NT>
static void tco_launch_rows(const TcPlan* tp, const TcRowsCand& c, const KDev* kd, int nk, cudaStream_t s) {
    TcOpParams p{};
    p.nk = nk;
    p.ns = tp->ns;
    p.ma = tp->ma;
    p.Dn = tp->Dn;
    p.kbps = c.kbps;
    p.splits = c.splits;
    p.atiles = tp->atiles;
    p.R = tp->Mp;
    p.S = c.S;
    p.fmt = tp->fmt;
    p.kd = kd;
    p.D = tp->Da;
    p.flag = tp->tflag;
    k_tc_opfwd<NT><<<dim3(tp->atiles, c.splits, nk), TCO_THREADS, c.smem, s>>>(tp->tbh, tp->tbl, tp->tah, tp->tal, p);
    TcRedParams r{};
    r.ns = tp->ns;
    r.ma = tp->ma;
    r.Dn = tp->Dn;
    r.kbps_a = c.kbps;
    r.splits_a = c.splits;
    r.Ra = tp->Mp;
    r.part = 2;
    r.inv_a = 1.0 / (tp->sA * tp->sC);
    r.kd = kd;
    r.Da = tp->Da;
    r.maxng = tp->maxng;
    k_tc_opred<<<tc_red_grid(r.part, tp->maxng, tp->ma, nk), 256, 0, s>>>(r);
}

template <int NT>
static void tco_launch_back(const TcPlan* tp, const TcRowsCand& c, const KDev* kd, int nk, cudaStream_t s,
                            int kofs = 0, int* flag = nullptr) {
    TcOpParams p{};
    p.kofs = kofs;
    p.nk = nk;
    p.ns = tp->ns;
    p.ma = tp->ma;
    p.Dn = tp->Dnb;
    p.kbps = c.kbps;
    p.splits = c.splits;
    p.atiles = tp->ttiles;
    p.R = tp->ttiles * TC_BM;
    p.S = c.S;
    p.nkb_fixed = tp->nkb_b;
    p.rows_ng = 1;
    p.fmt = tp->fmt;
    p.kd = kd;
    p.D = tp->Db;
    p.flag = flag ? flag : tp->tflag;
    p.nh = c.nh;
    if (c.nh > 1)  // column parts of 128: right-operand boxes of 128 rows
        k_tc_opfwd<128><<<dim3(tp->ttiles * c.nh, c.splits, nk), TCO_THREADS, c.smem, s>>>(tp->tzh2, tp->tzl2, tp->tabh,
                                                                                         tp->tabl, p);
    else
        k_tc_opfwd<NT><<<dim3(tp->ttiles, c.splits, nk), TCO_THREADS, c.smem, s>>>(tp->tzh, tp->tzl, tp->tabh, tp->tabl,
                                                                                  p);
    TcRedParams r{};
    r.ns = tp->ns;
    r.ma = tp->ma;
    r.part = 3;
    r.Dnb = tp->Dnb;
    r.kbps_b = c.kbps;
    r.splits_b = c.splits;
    r.nkb_b = tp->nkb_b;
    r.Rb = tp->ttiles * TC_BM;
    r.inv_b = 1.0 / (tp->sA * tp->sZ);
    r.kd = kd;
    r.Db = tp->Db;
    r.maxng = tp->maxng;
    k_tc_opred<<<tc_red_grid(r.part, tp->maxng, tp->ma, nk), 256, 0, s>>>(r);
}

static void tco_launch_back_any(const TcPlan* tp, const TcRowsCand& c, const KDev* kd, int nk, cudaStream_t s,
                                int kofs = 0, int* flag = nullptr) {
    switch (tp->NTb) {
#define RTD_TCO(n) \
    case n: tco_launch_back<n>(tp, c, kd, nk, s, kofs, flag); break;
        RTD_TCO(16) RTD_TCO(32) RTD_TCO(48) RTD_TCO(64) RTD_TCO(96) RTD_TCO(128) RTD_TCO(160) RTD_TCO(192)
        RTD_TCO(224) RTD_TCO(256)
#undef RTD_TCO
    }
}

// time the back-projection candidates and keep the fastest
static int tco_tune_back(TcPlan* tp, std::vector<TcRowsCand>& tb, const KDev* kd, int nk, cudaStream_t s) {
    if (tb.empty()) return 0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1;
    int best = 0;
    for (size_t i = 0; i < tb.size(); ++i) {
        tco_launch_back_any(tp, tb[i], kd, nk, s);
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r) tco_launch_back_any(tp, tb[i], kd, nk, s);
        cudaEventRecord(e1, s);
        float ms = 1e30f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) ms = 1e30f;
        tb[i].ms = ms;
        if (ms < tb[best].ms) best = (int)i;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int flag = 0;
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(&flag, tp->tflag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || flag)
        return -1;
    tp->S_b = tb[best].S;
    tp->kbps_b = tb[best].kbps;
    tp->splits_b = tb[best].splits;
    tp->nh_b = tb[best].nh;
    tp->smem_b = tb[best].smem;
    tp->ms_b = tb[best].ms / 3;
    tp->ncand += (int)tb.size();
    return 0;
}

// Candidate families for tests and measurements: RTTDDFT_TC_FAMILY in the
// environment holds comma-separated words that restrict the shapes the set-up
// autotuner times: "window" or "gather" (the interstitial table staged in
// shared memory or read through L1/L2), "fewslices" or "manyslices" (the
// largest or smallest K slice of the remaining shapes), "minstages" or
// "maxstages" (the fewest or most pipeline stages of the remaining shapes),
// "gen8" or "gen16" (8 or 16 generating warps in the interstitial launch;
// 16 only with the gathered table), "asmem" or "atmem" (its generated left
// operand in shared or tensor memory; tensor memory only with the gathered
// table), "bparts1" or "bparts2" (the back-projection's output columns in one
// part of up to 256 or in parts of 128; parts only above 128 columns).
// The restriction applies to the interstitial launch, the matching rows and
// the back-projection alike.  Unset: every shape is timed.
struct TcFamily {
    int route = 0;   // 1 window, 2 gather
    int slices = 0;  // 1 few (largest K slice), 2 many (smallest)
    int stages = 0;  // 1 min, 2 max
    int gen = 0;     // generating warps of the interstitial launch: 8 or 16
    int ta = 0;      // its left operand: 1 shared memory, 2 tensor memory
    int bparts = 0;  // back-projection output column parts: 1 or 2
};
static TcFamily tc_family_from_env() {
    TcFamily f;
    const char* v = getenv("RTTDDFT_TC_FAMILY");
    if (!v) return f;
    const std::string s(v);
    auto has = [&](const char* w) { return s.find(w) != std::string::npos; };
    f.route = has("window") ? 1 : (has("gather") ? 2 : 0);
    f.slices = has("fewslices") ? 1 : (has("manyslices") ? 2 : 0);
    f.stages = has("minstages") ? 1 : (has("maxstages") ? 2 : 0);
    f.gen = has("gen16") ? 16 : (has("gen8") ? 8 : 0);
    f.ta = has("atmem") ? 2 : (has("asmem") ? 1 : 0);
    f.bparts = has("bparts2") ? 2 : (has("bparts1") ? 1 : 0);
    return f;
}
template <typename C, typename KeyF>
static void tc_keep_extreme(std::vector<C>& v, int which, KeyF key) {
    if (!which || v.empty()) return;
    long best = key(v[0]);
    for (const C& c : v) best = which == 1 ? std::min(best, key(c)) : std::max(best, key(c));
    std::vector<C> out;
    for (const C& c : v)
        if (key(c) == best) out.push_back(c);
    v.swap(out);
}
static void tc_filter_family(const TcFamily& f, std::vector<TcToepCand>& tc, std::vector<TcRowsCand>& ta,
                             std::vector<TcRowsCand>& tb) {
    if (f.route) {
        std::vector<TcToepCand> out;
        for (const auto& c : tc)
            if ((f.route == 1) == (c.wn > 0)) out.push_back(c);
        tc.swap(out);
    }
    if (f.gen) {
        std::vector<TcToepCand> out;
        for (const auto& c : tc)
            if (c.gen == 32 * f.gen) out.push_back(c);
        tc.swap(out);
    }
    if (f.ta) {
        std::vector<TcToepCand> out;
        for (const auto& c : tc)
            if (c.ta == f.ta - 1) out.push_back(c);
        tc.swap(out);
    }
    if (f.bparts) {
        std::vector<TcRowsCand> out;
        for (const auto& c : tb)
            if (c.nh == f.bparts) out.push_back(c);
        tb.swap(out);
    }
    // few slices = the largest K slice (kbps): keep the maximum of kbps
    const int sl = f.slices == 1 ? 2 : (f.slices == 2 ? 1 : 0);
    tc_keep_extreme(tc, sl, [](const TcToepCand& c) { return (long)c.kbps; });
    tc_keep_extreme(ta, sl, [](const TcRowsCand& c) { return (long)c.kbps; });
    tc_keep_extreme(tb, sl, [](const TcRowsCand& c) { return (long)c.kbps; });
    tc_keep_extreme(tc, f.stages, [](const TcToepCand& c) { return (long)c.SA * 100 + c.SB; });
    tc_keep_extreme(ta, f.stages, [](const TcRowsCand& c) { return (long)c.S; });
    tc_keep_extreme(tb, f.stages, [](const TcRowsCand& c) { return (long)c.S; });
}

template <int NT>
static int tco_tune_t(TcPlan* tp, std::vector<TcToepCand>& tc, std::vector<TcRowsCand>& ta, const KDev* kd, int nk,
                      cudaStream_t s) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1;
    auto time_it = [&](auto&& launch) -> float {
        launch();
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r) launch();
        cudaEventRecord(e1, s);
        float ms = 1e30f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) ms = 1e30f;
        return ms;
    };
    int bt = 0;
    for (size_t i = 0; i < tc.size(); ++i) {
        tc[i].ms = time_it([&] { tco_launch_toep<NT>(tp, tc[i], kd, nk, s); });
        if (tc[i].ms < tc[bt].ms) bt = (int)i;
    }
    int ba = 0;
    for (size_t i = 0; i < ta.size(); ++i) {
        ta[i].ms = time_it([&] { tco_launch_rows<NT>(tp, ta[i], kd, nk, s); });
        if (ta[i].ms < ta[ba].ms) ba = (int)i;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int flag = 0;
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(&flag, tp->tflag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || flag)
        return -1;
    const TcToepCand& c = tc[bt];
    tp->kbps_t = c.kbps;
    tp->splits_t = c.splits;
    tp->SA = c.SA;
    tp->SB = c.SB;
    tp->wcap = c.wn;
    tp->gen_t = c.gen;
    tp->ta_t = c.ta;
    tp->smem_t = c.smem;
    tp->ms_t = c.ms / 3;
    if (!ta.empty()) {
        const TcRowsCand& r = ta[ba];
        tp->kbps_a = r.kbps;
        tp->splits_a = r.splits;
        tp->S_a = r.S;
        tp->smem_a = r.smem;
        tp->ms_a = r.ms / 3;
    }
    tp->ncand = (int)(tc.size() + ta.size());
    return 0;
}

static int tco_tune(TcPlan* tp, std::vector<TcToepCand>& tc, std::vector<TcRowsCand>& ta, const KDev* kd, int nk,
                    cudaStream_t s) {
    switch (tp->NT) {
#define RTD_TCO(n) \
    case n: return tco_tune_t<n>(tp, tc, ta, kd, nk, s);
        RTD_TCO(16) RTD_TCO(32) RTD_TCO(48) RTD_TCO(64) RTD_TCO(96) RTD_TCO(128) RTD_TCO(160) RTD_TCO(192)
        RTD_TCO(224) RTD_TCO(256)
#undef RTD_TCO
    }
    return -1;
}

int tc_plan_create(TcPlan** out, int nk, int ns, int ma, const int* ng, const int* const* glin_host,
                   const zd* const* at_dev, const zd* vtab, int nvt, int vt_center, const KDev* d_kd,
                   int fmt, double sa, double st, cudaStream_t s, std::string* why) {
    *out = nullptr;
    if (!get_encode()) {
        *why = "the driver has no tensor-map encoder";
        return RTTDDFT_ERR_UNSUPPORTED;
    }
    TcPlan* tp = new TcPlan();
    tp->nk = nk;
    tp->ns = ns;
    tp->ma = ma;
    tp->Dn = 2 * ns;
    tp->vt_center = vt_center;
    tp->fmt = fmt;
    if (!fmt) {
        // fp16: the matching coefficients and the table scaled to ~2^14 at their
        // largest entry, C (|c| <= 16) by 2^12 and Z (|z| <= 64) by 2^10
        tp->sA = sa;
        tp->sT = st;
        tp->sC = 4096.0;
        tp->sZ = 1024.0;
    }
    for (int nt : TCO_NTS)
        if (nt >= tp->Dn) {
            tp->NT = nt;
            break;
        }
    if (!tp->NT) {
        delete tp;
        *why = "the tensor-core form takes at most 128 states";
        return RTTDDFT_ERR_UNSUPPORTED;
    }
    int dev = 0, nsm = 148, smax = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int budget = smax - 512;
    int maxng = 0;
    for (int k = 0; k < nk; ++k) maxng = std::max(maxng, ng[k]);
    tp->maxng = maxng;
    const int nkb = (maxng + 31) / 32;
    tp->ttiles = (maxng + TC_BM - 1) / TC_BM;
    tp->atiles = (ma + TC_BM - 1) / TC_BM;
    const int A2 = 4 * TC_BM * TC_BK, B2 = 4 * tp->NT * TC_BK;  // hi + lo bytes of a stage
    // candidate shapes of the interstitial launch: K slices, generated stages SA,
    // copied stages SB, all that fit
    std::vector<TcToepCand> tc_c;
    {
        const int s0 = tco_best_splits(tp->ttiles, nk, nkb, nsm, 1);
        int last_kbps = -1;
        // K slices: from the cost model's choice, halving the blocks per slice down to
        // one; at most 8 slice sizes that fit, and partial outputs of at most 4 GB
        int tried = 0;
        for (int kbps = (nkb + s0 - 1) / s0; kbps >= 1 && tried < 8; kbps = (kbps == 1 ? 0 : (kbps + 1) / 2)) {
            if (kbps == last_kbps) break;
            last_kbps = kbps;
            const int sp = (nkb + kbps - 1) / kbps;
            if ((double)nk * sp * tp->ttiles * TC_BM * tp->Dn * 4.0 > 4.0e9) break;
            const int wn = tco_max_window(nk, ng, glin_host, kbps);
            bool any = false;
            for (int SA = 2; SA <= TCT_MAXSA; ++SA)
                for (int SB : {2, 4, 8, 16}) {
                    if (SB > TCT_MAXSB) continue;
                    const size_t need = 1024 + (size_t)SA * A2 + (size_t)SB * B2 + (size_t)kbps * 128 + (size_t)wn * 8;
                    if ((int)need <= budget) {
                        tc_c.push_back({kbps, sp, SA, SB, wn, 256, 0, need, 0.f});
                        any = true;
                    }
                }
            if (any) ++tried;
        }
        // table gathered through L1/L2: no window, so any K slice fits
        last_kbps = -1;
        for (int kbps = (nkb + s0 - 1) / s0, n = 0; kbps >= 1 && n < 3; kbps = (kbps + 1) / 2, ++n) {
            if (kbps == last_kbps) break;
            last_kbps = kbps;
            const int sp = (nkb + kbps - 1) / kbps;
            if ((double)nk * sp * tp->ttiles * TC_BM * tp->Dn * 4.0 > 4.0e9) break;
            for (int SA = 2; SA <= TCT_MAXSA; ++SA)
                for (int SB : {2, 4, 8}) {
                    const size_t need = 1024 + (size_t)SA * A2 + (size_t)SB * B2 + (size_t)kbps * 128;
                    if ((int)need <= budget)
                        for (int gen : {256, 512}) tc_c.push_back({kbps, sp, SA, SB, 0, gen, 0, need, 0.f});
                    // left operand in tensor memory: no shared-memory stages for it; at least
                    // 120 KB requested so that one block holds an SM (it allocates all 512
                    // tensor-memory columns)
                    const size_t need_ta = std::max<size_t>(1024 + (size_t)SB * B2 + (size_t)kbps * 128, 120 * 1024);
                    if ((int)need_ta <= budget)
                        for (int gen : {256, 512}) tc_c.push_back({kbps, sp, SA, SB, 0, gen, 1, need_ta, 0.f});
                }
            if (kbps == 1) break;
        }
    }
    if (tc_c.empty()) {
        delete tp;
        *why = "the interstitial table window of one K block does not fit in shared memory";
        return RTTDDFT_ERR_UNSUPPORTED;
    }
    // matching rows: K slices and stages
    std::vector<TcRowsCand> ta_c;
    if (tp->atiles > 0) {
        const int s0 = tco_best_splits(tp->atiles, nk, nkb, nsm, 1);
        int last_kbps = -1;
        for (int mult = 1; mult <= 8; mult *= 2) {
            const int sp = std::min(nkb, s0 * mult);
            const int kbps = (nkb + sp - 1) / sp;
            if (kbps == last_kbps) continue;
            last_kbps = kbps;
            for (int S = 2; S <= TCO_MAXS; ++S) {
                const size_t need = 1024 + (size_t)S * (A2 + B2) + (size_t)kbps * 128;
                if ((int)need <= budget) ta_c.push_back({kbps, (nkb + kbps - 1) / kbps, S, need, 0.f, 1});
            }
        }
    }
    int max_sp_t = 0, max_sp_a = 1;
    size_t max_sm_t = 0, max_sm_a = 0;
    for (auto& c : tc_c) {
        max_sp_t = std::max(max_sp_t, c.splits);
        max_sm_t = std::max(max_sm_t, c.smem);
    }
    for (auto& c : ta_c) {
        max_sp_a = std::max(max_sp_a, c.splits);
        max_sm_a = std::max(max_sm_a, c.smem);
    }
    tp->Kp = nkb * TC_BK;
    tp->Rp = tp->NT;
    tp->Mp = std::max(1, tp->atiles) * TC_BM;
    const size_t nbh = (size_t)nk * tp->Rp * tp->Kp, nah = (size_t)nk * tp->Mp * tp->Kp;
    const size_t ndt = (size_t)nk * max_sp_t * tp->ttiles * TC_BM * tp->Dn;
    const size_t nda = (size_t)nk * max_sp_a * tp->Mp * tp->Dn;
    if (cudaMalloc(&tp->bh, nbh * 2) != cudaSuccess || cudaMalloc(&tp->bl, nbh * 2) != cudaSuccess ||
        cudaMalloc(&tp->ah, nah * 2) != cudaSuccess || cudaMalloc(&tp->al, nah * 2) != cudaSuccess ||
        cudaMalloc(&tp->Dt, ndt * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&tp->Da, nda * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&tp->tabs, (size_t)std::max(1, nvt) * sizeof(uint2)) != cudaSuccess ||
        cudaMalloc(&tp->tflag, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        tc_plan_destroy(tp);
        *why = "out of device memory for the tensor-core operands";
        return RTTDDFT_ERR_OOM;
    }
    cudaMemsetAsync(tp->bh, 0, nbh * 2, s);
    cudaMemsetAsync(tp->bl, 0, nbh * 2, s);
    cudaMemsetAsync(tp->ah, 0, nah * 2, s);
    cudaMemsetAsync(tp->al, 0, nah * 2, s);
    cudaMemsetAsync(tp->tflag, 0, sizeof(int), s);
    if (nvt > 0) k_tc_split_table<<<(nvt + 255) / 256, 256, 0, s>>>(vtab, tp->tabs, nvt, tp->fmt, tp->sT, tp->tflag);
    for (int k = 0; k < nk && ma > 0; ++k) {
        const size_t n = (size_t)ma * ng[k];
        k_tc_pack_at<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(at_dev[k], ng[k], ma, tp->Kp, tp->Mp, k, tp->ah,
                                                                 tp->al, tp->fmt, tp->sA, tp->tflag);
    }
    int e = tc_tmap3(&tp->tbh, tp->bh, tp->Kp, tp->Rp, nk, tp->NT) | tc_tmap3(&tp->tbl, tp->bl, tp->Kp, tp->Rp, nk, tp->NT) |
            tc_tmap3(&tp->tah, tp->ah, tp->Kp, tp->Mp, nk, TC_BM) | tc_tmap3(&tp->tal, tp->al, tp->Kp, tp->Mp, nk, TC_BM);
    // back-projection Y_G += A^H [hQ | oQ] (4 ns real output columns, K = matching rows)
    std::vector<TcRowsCand> tb_c;
    if (ma > 0 && 4 * ns <= 256) {
        tp->Dnb = 4 * ns;
        for (int nt : TCO_NTS)
            if (nt >= tp->Dnb) {
                tp->NTb = nt;
                break;
            }
        tp->nkb_b = (ma + 31) / 32;
        tp->Kpb = tp->nkb_b * TC_BK;
        tp->Rpb = tp->NTb;
        const int Bb2 = 4 * tp->NTb * TC_BK;
        const int s0 = tco_best_splits(tp->ttiles, nk, tp->nkb_b, nsm, 1);
        int last_kbps = -1;
        for (int mult = 1; mult <= 8; mult *= 2) {
            const int sp = std::min(tp->nkb_b, s0 * mult);
            const int kbps = (tp->nkb_b + sp - 1) / sp;
            if (kbps == last_kbps) continue;
            last_kbps = kbps;
            const int spl = (tp->nkb_b + kbps - 1) / kbps;
            if ((double)nk * spl * tp->ttiles * TC_BM * tp->Dnb * 4.0 > 4.0e9) break;
            for (int S = 2; S <= TCO_MAXS; ++S) {
                const size_t need = 1024 + (size_t)S * (A2 + Bb2);
                if ((int)need <= budget) tb_c.push_back({kbps, spl, S, need, 0.f, 1});
                // two column parts of 128 (right-operand boxes of 128 rows): smaller
                // stages, more of them; the parts of a row tile read the same left-
                // operand blocks at about the same time, so the second read is an L2 hit
                if (tp->NTb > 128) {
                    const size_t need2 = 1024 + (size_t)S * (A2 + 4 * 128 * TC_BK);
                    if ((int)need2 <= budget) tb_c.push_back({kbps, spl, S, need2, 0.f, 2});
                }
            }
        }
        int max_sp_b = 1;
        size_t max_sm_b = 1024;
        for (auto& c : tb_c) {
            max_sp_b = std::max(max_sp_b, c.splits);
            max_sm_b = std::max(max_sm_b, c.smem);
        }
        const size_t nzb = (size_t)nk * tp->Rpb * tp->Kpb, nab = (size_t)nk * tp->ttiles * TC_BM * tp->Kpb;
        const size_t ndb = (size_t)nk * max_sp_b * tp->ttiles * TC_BM * tp->Dnb;
        if (tb_c.empty() || cudaMalloc(&tp->zh, nzb * 2) != cudaSuccess || cudaMalloc(&tp->zl, nzb * 2) != cudaSuccess ||
            cudaMalloc(&tp->abh, nab * 2) != cudaSuccess || cudaMalloc(&tp->abl, nab * 2) != cudaSuccess ||
            cudaMalloc(&tp->Db, ndb * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            tc_plan_destroy(tp);
            *why = "out of device memory for the back-projection operands";
            return RTTDDFT_ERR_OOM;
        }
        cudaMemsetAsync(tp->zh, 0, nzb * 2, s);
        cudaMemsetAsync(tp->zl, 0, nzb * 2, s);
        cudaMemsetAsync(tp->abh, 0, nab * 2, s);
        cudaMemsetAsync(tp->abl, 0, nab * 2, s);
        for (int k = 0; k < nk; ++k) {
            const size_t n = (size_t)ma * ng[k];
            k_tc_pack_atb<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(at_dev[k], ng[k], ma, tp->Kpb, tp->ttiles * TC_BM,
                                                                       k, tp->abh, tp->abl, tp->fmt, tp->sA, tp->tflag);
        }
        e |= tc_tmap3(&tp->tzh, tp->zh, tp->Kpb, tp->Rpb, nk, tp->NTb) |
             tc_tmap3(&tp->tzl, tp->zl, tp->Kpb, tp->Rpb, nk, tp->NTb) |
             (tp->NTb > 128 ? (tc_tmap3(&tp->tzh2, tp->zh, tp->Kpb, tp->Rpb, nk, 128) |
                               tc_tmap3(&tp->tzl2, tp->zl, tp->Kpb, tp->Rpb, nk, 128))
                            : 0) |
             tc_tmap3(&tp->tabh, tp->abh, tp->Kpb, (uint64_t)tp->ttiles * TC_BM, nk, TC_BM) |
             tc_tmap3(&tp->tabl, tp->abl, tp->Kpb, (uint64_t)tp->ttiles * TC_BM, nk, TC_BM);
        cudaError_t cb = cudaSuccess;
        switch (tp->NTb) {
#define RTD_TCO(n) \
    case n: cb = raise_smem((const void*)k_tc_opfwd<n>, (int)std::max(max_sm_b, std::max(max_sm_a, (size_t)1024))); break;
            RTD_TCO(16) RTD_TCO(32) RTD_TCO(48) RTD_TCO(64) RTD_TCO(96) RTD_TCO(128) RTD_TCO(160) RTD_TCO(192)
            RTD_TCO(224) RTD_TCO(256)
#undef RTD_TCO
        }
        if (cb == cudaSuccess && tp->NTb > 128)
            cb = raise_smem((const void*)k_tc_opfwd<128>, (int)std::max(max_sm_b, std::max(max_sm_a, (size_t)1024)));
        if (cb != cudaSuccess) e |= 1;
    }
    cudaError_t ce = cudaSuccess;
    switch (tp->NT) {
#define RTD_TCO(n) \
    case n: ce = tco_set_smem<n>((int)std::max(max_sm_a, (size_t)1024), (int)max_sm_t); break;
        RTD_TCO(16) RTD_TCO(32) RTD_TCO(48) RTD_TCO(64) RTD_TCO(96) RTD_TCO(128) RTD_TCO(160) RTD_TCO(192)
        RTD_TCO(224) RTD_TCO(256)
#undef RTD_TCO
    }
    if (e || ce != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        tc_plan_destroy(tp);
        *why = "tensor-core operand set-up failed";
        return RTTDDFT_ERR_CUDA;
    }
    // autotune: time every candidate on these operands (3 launches after one
    // warm-up) and keep the fastest
    tc_filter_family(tc_family_from_env(), tc_c, ta_c, tb_c);
    if (tc_c.empty() || (tp->atiles > 0 && ta_c.empty()) || (tp->Dnb > 0 && tb_c.empty())) {
        tc_plan_destroy(tp);
        *why = "no tensor-core launch shape of the family in RTTDDFT_TC_FAMILY fits";
        return RTTDDFT_ERR_UNSUPPORTED;
    }
    int ti = tco_tune(tp, tc_c, ta_c, d_kd, nk, s);
    if (!ti) ti = tco_tune_back(tp, tb_c, d_kd, nk, s);
    if (ti) {
        tc_plan_destroy(tp);
        *why = "tensor-core autotuning failed";
        return RTTDDFT_ERR_CUDA;
    }
    *out = tp;
    return RTTDDFT_OK;
}

static TcOpParams tco_rows_params(const TcPlan* tp, const StepArgs& a) {
    TcOpParams p{};
    p.nk = a.nk;
    p.ns = tp->ns;
    p.ma = tp->ma;
    p.Dn = tp->Dn;
    p.kbps = tp->kbps_a;
    p.splits = tp->splits_a;
    p.atiles = tp->atiles;
    p.R = tp->Mp;
    p.S = tp->S_a;
    p.kofs = a.kofs;
    p.fmt = tp->fmt;
    p.kd = a.kd;
    p.D = tp->Da;
    p.flag = a.flag;
    return p;
}

static TcToepParams tco_toep_params(const TcPlan* tp, const StepArgs& a) {
    TcToepParams p{};
    p.nk = a.nk;
    p.Dn = tp->Dn;
    p.kbps = tp->kbps_t;
    p.splits = tp->splits_t;
    p.ttiles = tp->ttiles;
    p.wcap = tp->wcap;
    p.vt_center = tp->vt_center;
    p.SA = tp->SA;
    p.SB = tp->SB;
    p.fmt = tp->fmt;
    p.kd = a.kd;
    p.tab = a.dv_on ? a.vsteps : tp->tabs;
    p.D = tp->Dt;
    p.flag = a.flag;
    return p;
}

void launch_tc_pack(const TcPlan* tp, const StepArgs& a, cudaStream_t s) {
    dim3 g((tp->ns * tp->maxng + 255) / 256, 1, a.nk);
    k_tc_pack_c<<<g, 256, 0, s>>>(a.kd, tp->ns, tp->Kp, tp->Rp, tp->bh, tp->bl, tp->fmt, tp->sC, a.flag);
}

int launch_tc_operator(const TcPlan* tp, const StepArgs& a, cudaStream_t s, bool rows_only) {
    const TcToepParams pt = tco_toep_params(tp, a);
    const TcOpParams pa = tco_rows_params(tp, a);
    dim3 gt(tp->ttiles, tp->splits_t, a.nk);
    dim3 ga(tp->atiles, tp->splits_a, a.nk);
    switch (tp->NT) {
#define RTD_TCO(n)                                                                                    \
    case n:                                                                                           \
        if (rows_only) {                                                                              \
        } else {                                                                                      \
            toep_variant<n>(tp->wcap, tp->gen_t, tp->ta_t, gt, tp->smem_t, s, tp->tbh, tp->tbl, pt);      \
        }                                                                                             \
        if (tp->atiles > 0) k_tc_opfwd<n><<<ga, TCO_THREADS, tp->smem_a, s>>>(tp->tbh, tp->tbl, tp->tah, tp->tal, pa); \
        break;
        RTD_TCO(16) RTD_TCO(32) RTD_TCO(48) RTD_TCO(64) RTD_TCO(96) RTD_TCO(128) RTD_TCO(160) RTD_TCO(192)
        RTD_TCO(224) RTD_TCO(256)
#undef RTD_TCO
    }
    return (rows_only ? 0 : 1) + (tp->atiles > 0 ? 1 : 0);
}

bool tc_has_back(const TcPlan* tp) { return tp && tp->NTb > 0; }

int launch_tc_back(const TcPlan* tp, const StepArgs& a, cudaStream_t s) {
    dim3 gz((2 * tp->ns * tp->ma + 255) / 256, 1, a.nk);
    k_tc_pack_z<<<gz, 256, 0, s>>>(a.kd, tp->ns, tp->ma, tp->Kpb, tp->Rpb, tp->zh, tp->zl, tp->fmt, tp->sZ, a.flag);
    TcRowsCand c{tp->kbps_b, tp->splits_b, tp->S_b, tp->smem_b, 0.f, tp->nh_b};
    tco_launch_back_any(tp, c, a.kd, a.nk, s, a.kofs, a.flag);  // single-k calls: left operand of k-point kofs
    return 3;
}

void launch_tc_reduce(const TcPlan* tp, const StepArgs& a, cudaStream_t s, bool rows_only) {
    TcRedParams p{};
    p.ns = tp->ns;
    p.ma = tp->ma;
    p.Dn = tp->Dn;
    p.kbps_t = tp->kbps_t;
    p.splits_t = tp->splits_t;
    p.kbps_a = tp->kbps_a;
    p.splits_a = tp->splits_a;
    p.Rt = tp->ttiles * TC_BM;
    p.Ra = tp->Mp;
    p.part = rows_only ? 2 : 0;
    p.inv_t = 1.0 / (tp->sT * tp->sC);
    p.inv_a = 1.0 / (tp->sA * tp->sC);
    p.kd = a.kd;
    p.Dt = tp->Dt;
    p.Da = tp->Da;
    p.maxng = tp->maxng;
    if (rows_only && tp->ma == 0) return;
    k_tc_opred<<<tc_red_grid(p.part, tp->maxng, tp->ma, a.nk), 256, 0, s>>>(p);
}

void tc_plan_info(const TcPlan* tp, int* v) {
    v[0] = tp->NT;
    v[1] = tp->SA * 100 + tp->SB;
    v[2] = tp->kbps_t;
    v[3] = tp->splits_t;
    v[4] = tp->wcap;
    v[5] = (int)tp->smem_t;
    v[6] = tp->ncand;
    v[7] = (int)(tp->ms_t * 1e6f);  // ns
    v[8] = (int)(tp->ms_a * 1e6f);
    v[9] = tp->gen_t;
    v[10] = tp->ta_t;
    v[11] = tp->NTb > 0 ? tp->nh_b : 0;
}

double tc_table_scale(const TcPlan* tp) { return tp ? tp->sT : 1.0; }
int tc_format(const TcPlan* tp) { return tp ? tp->fmt : 1; }

// ------------------------------------------------------------ potential-change rebuild
// CC_G packed per column tile: rows [j NTV, j NTV + h_j) hold [Re CC | -Im CC] of the
// tile's h_j columns, rows [j NTV + h_j, j NTV + 2 h_j) hold [Im CC | Re CC].
#define TC_DV_NT 256
__global__ void k_tc_pack_cc(const zd* __restrict__ caux, int nb, int ng, int naux, int Kp, int rows, int k,
                             unsigned short* __restrict__ bh, unsigned short* __restrict__ bl, int fmt, double sc,
                             int* flag) {
    const size_t e = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (e >= (size_t)naux * ng) return;
    const int gp = (int)(e % ng), col = (int)(e / ng);
    const int j = col / (TC_DV_NT / 2), cl = col % (TC_DV_NT / 2);
    const int h = min(TC_DV_NT / 2, naux - j * (TC_DV_NT / 2));
    const zd c = caux[gp + (size_t)col * nb];
    const int kb = gp >> 5, o = gp & 31;
    const size_t re_row = ((size_t)k * rows + (size_t)j * TC_DV_NT + cl) * Kp + (size_t)kb * 64;
    const size_t im_row = ((size_t)k * rows + (size_t)j * TC_DV_NT + h + cl) * Kp + (size_t)kb * 64;
    put16(c.x, fmt, sc, bh, bl, re_row + o, flag);
    put16(c.x, fmt, sc, bh, bl, im_row + 32 + o, flag);
    put16(c.y, fmt, sc, bh, bl, im_row + o, flag);
    put16(-c.y, fmt, sc, bh, bl, re_row + 32 + o, flag);
}

// T[G + (c0 + c) ng] = s sum over slices (tile of h columns); T is the per-k
// buffer of the descriptor's B operand (dv[k].X of the Toeplitz descriptor)
struct TcDvRedParams {
    int splits, kbps, Rt, h, c0;
    double inv;  // 1 / (scale of CC_G x scale of the table)
    const KDev* kd;
    const ToepDesc* td;
    const float* D;
    const DevState* st;
};
__global__ void __launch_bounds__(256) k_tc_dvred(TcDvRedParams p) {
    __shared__ double tile[TC_RT][257];
    const int k = blockIdx.z;
    const KDev& K = p.kd[k];
    const int ng = K.ng, nkb = (ng + 31) >> 5;
    const int row0 = blockIdx.x * TC_RT;
    if (row0 >= ng) return;
    const int nsp = min(p.splits, (nkb + p.kbps - 1) / p.kbps);
    tc_red_tile(p.D + (size_t)k * p.splits * p.Rt * TC_DV_NT, (size_t)p.Rt * TC_DV_NT, nsp, TC_DV_NT, p.h, row0, ng,
                p.st->cur_s * p.inv, p.td[k].Y + (size_t)p.c0 * ng, ng, tile);
}

// Set-up of the rebuild operands (at the first rttddft_set_dv): CC_G packed,
// the dV~ table pre-split, the partial-output buffer.
int tc_dv_prepare(TcPlan* tp, const zd* const* caux_dev, const int* nb, const int* ng, int naux, int nvt,
                  cudaStream_t s, std::string* why) {
    if (tp->dv_ready) return RTTDDFT_OK;
    tp->naux = naux;
    tp->dv_tiles = (naux + TC_DV_NT / 2 - 1) / (TC_DV_NT / 2);
    const int nkb = tp->Kp / TC_BK;
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int smax = 0;
    cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int sp = std::max(1, std::min(nkb, (2 * nsm + tp->ttiles * tp->nk - 1) / (tp->ttiles * tp->nk)));
    // two stages of each operand plus 128 bytes per K block of a slice: cap the
    // slice so that the block fits in the opt-in shared memory
    const size_t fixed = 1024 + (size_t)2 * 4 * TC_BM * TC_BK + (size_t)2 * 4 * TC_DV_NT * TC_BK;
    const int kb_cap = (int)std::max<long>(1, ((long)smax - 512 - (long)fixed) / 128);
    tp->dv_kbps = std::min((nkb + sp - 1) / sp, kb_cap);
    tp->dv_splits = (nkb + tp->dv_kbps - 1) / tp->dv_kbps;
    tp->dv_smem = fixed + (size_t)tp->dv_kbps * 128;
    const int rows = tp->dv_tiles * TC_DV_NT;
    const size_t ncc = (size_t)tp->nk * rows * tp->Kp;
    const size_t nd = (size_t)tp->nk * tp->dv_splits * tp->ttiles * TC_BM * TC_DV_NT;
    if (cudaMalloc(&tp->cch, ncc * 2) != cudaSuccess || cudaMalloc(&tp->ccl, ncc * 2) != cudaSuccess ||
        cudaMalloc(&tp->dvtabs, (size_t)std::max(1, nvt) * sizeof(uint2)) != cudaSuccess ||
        cudaMalloc(&tp->Dd, nd * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        *why = "out of device memory for the potential-change operands";
        return RTTDDFT_ERR_OOM;
    }
    cudaMemsetAsync(tp->cch, 0, ncc * 2, s);
    cudaMemsetAsync(tp->ccl, 0, ncc * 2, s);
    // fp16 form: the plane-wave rows of an S-orthonormal CC have |c| <= 1 (S >= I on
    // them), so 2^14 keeps every packed value inside the fp16 range
    tp->dv_sc = tp->fmt ? 1.0 : 16384.0;
    for (int k = 0; k < tp->nk; ++k) {
        const size_t n = (size_t)naux * ng[k];
        k_tc_pack_cc<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(caux_dev[k], nb[k], ng[k], naux, tp->Kp, rows, k,
                                                                 tp->cch, tp->ccl, tp->fmt, tp->dv_sc, tp->tflag);
    }
    int e = tc_tmap3(&tp->tch, tp->cch, tp->Kp, rows, tp->nk, TC_DV_NT) |
            tc_tmap3(&tp->tcl, tp->ccl, tp->Kp, rows, tp->nk, TC_DV_NT);
    const cudaError_t ce = raise_smem((const void*)k_tc_toep<TC_DV_NT, true, 256, false>, (int)tp->dv_smem);
    if (e || ce != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        *why = "potential-change operand set-up failed";
        return RTTDDFT_ERR_CUDA;
    }
    tp->dv_ready = 1;
    return RTTDDFT_OK;
}

// the pre-split dV~ table (every rttddft_set_dv); vmax: its largest |Re|, |Im|
// (the fp16 form scales it by a power of two to about 2^14)
void tc_dv_set_table(TcPlan* tp, const zd* dvtab, int nvt, double vmax, cudaStream_t s) {
    tp->dv_st = 1.0;
    if (!tp->fmt && vmax > 0.0) tp->dv_st = std::ldexp(1.0, (int)std::floor(std::log2(16384.0 / vmax)));
    if (nvt > 0)
        k_tc_split_table<<<(nvt + 255) / 256, 256, 0, s>>>(dvtab, tp->dvtabs, nvt, tp->fmt, tp->dv_st, tp->tflag);
}

bool tc_dv_ready(const TcPlan* tp) { return tp && tp->dv_ready; }
int tc_dv_tiles(const TcPlan* tp) { return tp ? tp->dv_tiles : 0; }

// T = s dV~ * CC_G for every column tile (into the Toeplitz descriptors' Y)
void launch_tc_dv_toeplitz(const TcPlan* tp, const StepArgs& a, const ToepDesc* td, cudaStream_t s) {
    TcToepParams p{};
    p.nk = a.nk;
    p.Dn = TC_DV_NT;
    p.kbps = tp->dv_kbps;
    p.splits = tp->dv_splits;
    p.ttiles = tp->ttiles;
    p.wcap = 0;
    p.vt_center = tp->vt_center;
    p.SA = 2;
    p.SB = 2;
    p.fmt = tp->fmt;
    p.kd = a.kd;
    p.tab = tp->dvtabs;
    p.D = tp->Dd;
    p.flag = a.flag;
    for (int j = 0; j < tp->dv_tiles; ++j) {
        p.brow0 = j * TC_DV_NT;
        k_tc_toep<TC_DV_NT, true, 256, false><<<dim3(tp->ttiles, tp->dv_splits, a.nk), 256 + 64, tp->dv_smem, s>>>(tp->tch,
                                                                                                         tp->tcl, p);
        TcDvRedParams r{};
        r.splits = tp->dv_splits;
        r.kbps = tp->dv_kbps;
        r.Rt = tp->ttiles * TC_BM;
        r.c0 = j * (TC_DV_NT / 2);
        r.inv = 1.0 / (tp->dv_sc * tp->dv_st);
        r.h = std::min(TC_DV_NT / 2, tp->naux - r.c0);
        r.kd = a.kd;
        r.td = td;
        r.D = tp->Dd;
        r.st = a.st;
        k_tc_dvred<<<dim3((tp->maxng + TC_RT - 1) / TC_RT, 1, a.nk), 256, 0, s>>>(r);
    }
}

// ------------------------------------------------------------ products with the auxiliary basis
// Expansion C = CC theta (Eq. approximation_coefficients) and projection
// theta~ = CC^H (S C) (Eq. evolution_of_projection_coeff) as split-BF16
// tensor-core products on the matching-row pipeline (k_tc_opfwd).  CC is
// split and packed once at set-up as the left operand of both: its rows with
// K over the auxiliary vectors (expansion), and the rows of CC^H with K over
// the basis rows (projection).  The right operand, theta or the S C columns
// of the operator pass, is packed every step.
struct TcCC {
    int nk = 0, naux = 0, ns = 0, NT = 0, Dn = 0, maxnb = 0;
    int Mp_e = 0, Kp_e = 0, nkb_e = 0, tiles_e = 0;
    int Mp_p = 0, Kp_p = 0, nkb_p = 0, tiles_p = 0, kbps_p = 0, splits_p = 0;
    int S = 2;
    size_t smem = 0;
    unsigned short *aeh = nullptr, *ael = nullptr, *aph = nullptr, *apl = nullptr;
    unsigned short *beh = nullptr, *bel = nullptr, *bph = nullptr, *bpl = nullptr;
    float *De = nullptr, *Dp = nullptr;
    CUtensorMap taeh, tael, taph, tapl, tbeh, tbel, tbph, tbpl;
};

void tc_cc_destroy(TcCC* t) {
    if (!t) return;
    for (void* q : {(void*)t->aeh, (void*)t->ael, (void*)t->aph, (void*)t->apl, (void*)t->beh, (void*)t->bel,
                    (void*)t->bph, (void*)t->bpl, (void*)t->De, (void*)t->Dp})
        cudaFree(q);
    delete t;
}

// left operands from CC (nb x naux, column-major): the expansion's rows b with
// K over i, the projection's rows i (of CC^H) with K over b
__global__ void k_tc_pack_cce(const zd* __restrict__ cc, int nb, int naux, int Kp, int Mp, int k,
                              unsigned short* __restrict__ ah, unsigned short* __restrict__ al, int* flag) {
    const size_t e = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (e >= (size_t)nb * naux) return;
    const int b = (int)(e % nb), i = (int)(e / nb);
    const zd v = cc[e];
    const size_t row = ((size_t)k * Mp + b) * Kp + (size_t)(i >> 5) * 64 + (i & 31);
    put16(v.x, 1, 1.0, ah, al, row, flag);
    put16(v.y, 1, 1.0, ah, al, row + 32, flag);
}
__global__ void k_tc_pack_ccp(const zd* __restrict__ cc, int nb, int naux, int Kp, int Mp, int k,
                              unsigned short* __restrict__ ah, unsigned short* __restrict__ al, int* flag) {
    const size_t e = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (e >= (size_t)nb * naux) return;
    const int b = (int)(e % nb), i = (int)(e / nb);
    const zd v = cc[e];
    const size_t row = ((size_t)k * Mp + i) * Kp + (size_t)(b >> 5) * 64 + (b & 31);
    put16(v.x, 1, 1.0, ah, al, row, flag);
    put16(-v.y, 1, 1.0, ah, al, row + 32, flag);
}
// right operand of a step: theta (mode 0, naux rows) or S C (mode 1, the S
// half of [HC | SC], nb rows); rows c < ns hold [Re x | -Im x], rows ns + c
// hold [Im x | Re x] over K
__global__ void k_tc_pack_cols(const KDev* __restrict__ kd, int mode, int ns, int naux, int maxr, int Kp, int Rp,
                               unsigned short* __restrict__ bh, unsigned short* __restrict__ bl, int* flag) {
    const int k = blockIdx.z;
    const KDev& K = kd[k];
    const int nr = mode ? K.nb : naux;
    const int e = blockIdx.x * 256 + threadIdx.x;
    if (e >= maxr * ns) return;
    const int r = e % maxr, c = e / maxr;
    if (r >= nr) return;
    const zd x = mode ? K.Y[(size_t)(ns + c) * K.nb + r] : K.theta[r + (size_t)c * naux];
    const int kb = r >> 5, o = r & 31;
    const size_t re_row = ((size_t)k * Rp + c) * Kp + (size_t)kb * 64;
    const size_t im_row = ((size_t)k * Rp + ns + c) * Kp + (size_t)kb * 64;
    put16(x.x, 1, 1.0, bh, bl, re_row + o, flag);
    put16(x.x, 1, 1.0, bh, bl, im_row + 32 + o, flag);
    put16(x.y, 1, 1.0, bh, bl, im_row + o, flag);
    put16(-x.y, 1, 1.0, bh, bl, re_row + 32 + o, flag);
}
// split-K sums: the expansion into K.C (mode 0), the projection into the
// single-slice projection partials that the post kernel finishes (mode 1)
struct TcCCRed {
    int mode, ns, naux, Dn, R, splits, kbps;
    const KDev* kd;
    const float* D;
    zd* part;
};
__global__ void __launch_bounds__(256) k_tc_ccred(TcCCRed p) {
    __shared__ double tile[TC_RT][257];
    const int k = blockIdx.z;
    const KDev& K = p.kd[k];
    const int row0 = blockIdx.x * TC_RT;
    const int nrow = p.mode ? p.naux : K.nb;
    if (row0 >= nrow) return;
    const int nsp = p.mode ? min(p.splits, (((K.nb + 31) >> 5) + p.kbps - 1) / p.kbps) : 1;
    zd* out = p.mode ? p.part + (size_t)k * p.naux * p.ns : K.C;
    tc_red_tile(p.D + (size_t)k * p.splits * p.R * p.Dn, (size_t)p.R * p.Dn, nsp, p.Dn, p.ns, row0, nrow, 1.0, out,
                p.mode ? p.naux : K.nb, tile);
}

int tc_cc_create(TcCC** out, int nk, int naux, int ns, const int* nb, const zd* const* cc_dev, int* flag,
                 cudaStream_t s, std::string* why) {
    *out = nullptr;
    if (!get_encode()) {
        *why = "the driver has no tensor-map encoder";
        return RTTDDFT_ERR_UNSUPPORTED;
    }
    TcCC* t = new TcCC();
    t->nk = nk;
    t->naux = naux;
    t->ns = ns;
    t->Dn = 2 * ns;
    for (int nt : TCO_NTS)
        if (nt >= t->Dn) {
            t->NT = nt;
            break;
        }
    if (!t->NT || t->NT > 128) {
        delete t;
        *why = "the tensor-core products with the auxiliary basis take at most 64 states";
        return RTTDDFT_ERR_UNSUPPORTED;
    }
    for (int k = 0; k < nk; ++k) t->maxnb = std::max(t->maxnb, nb[k]);
    int dev = 0, nsm = 148, smax = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    t->nkb_e = (naux + 31) / 32;
    t->Kp_e = t->nkb_e * TC_BK;
    t->tiles_e = (t->maxnb + TC_BM - 1) / TC_BM;
    t->Mp_e = t->tiles_e * TC_BM;
    t->nkb_p = (t->maxnb + 31) / 32;
    t->Kp_p = t->nkb_p * TC_BK;
    t->tiles_p = (naux + TC_BM - 1) / TC_BM;
    t->Mp_p = t->tiles_p * TC_BM;
    {
        // projection: K slices so that about two blocks per SM work
        int sp = std::max(1, std::min(t->nkb_p, (2 * nsm + t->tiles_p * nk - 1) / (t->tiles_p * nk)));
        t->kbps_p = (t->nkb_p + sp - 1) / sp;
        t->splits_p = (t->nkb_p + t->kbps_p - 1) / t->kbps_p;
    }
    const size_t stage = (size_t)2 * TC_BM * TC_BK * 2 + (size_t)2 * t->NT * TC_BK * 2;
    t->S = 4;
    while (t->S > 2 && 1024 + t->S * stage > (size_t)smax - 512) --t->S;
    t->smem = 1024 + t->S * stage;
    const size_t nae = (size_t)nk * t->Mp_e * t->Kp_e, nap = (size_t)nk * t->Mp_p * t->Kp_p;
    const size_t nbe = (size_t)nk * t->NT * t->Kp_e, nbp = (size_t)nk * t->NT * t->Kp_p;
    const size_t nde = (size_t)nk * t->Mp_e * t->Dn, ndp = (size_t)nk * t->splits_p * t->Mp_p * t->Dn;
    if (cudaMalloc(&t->aeh, nae * 2) != cudaSuccess || cudaMalloc(&t->ael, nae * 2) != cudaSuccess ||
        cudaMalloc(&t->aph, nap * 2) != cudaSuccess || cudaMalloc(&t->apl, nap * 2) != cudaSuccess ||
        cudaMalloc(&t->beh, nbe * 2) != cudaSuccess || cudaMalloc(&t->bel, nbe * 2) != cudaSuccess ||
        cudaMalloc(&t->bph, nbp * 2) != cudaSuccess || cudaMalloc(&t->bpl, nbp * 2) != cudaSuccess ||
        cudaMalloc(&t->De, nde * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&t->Dp, ndp * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        tc_cc_destroy(t);
        *why = "out of device memory for the tensor-core products with the auxiliary basis";
        return RTTDDFT_ERR_OOM;
    }
    for (auto pr : {std::make_pair((void*)t->aeh, nae), std::make_pair((void*)t->ael, nae),
                    std::make_pair((void*)t->aph, nap), std::make_pair((void*)t->apl, nap),
                    std::make_pair((void*)t->beh, nbe), std::make_pair((void*)t->bel, nbe),
                    std::make_pair((void*)t->bph, nbp), std::make_pair((void*)t->bpl, nbp)})
        cudaMemsetAsync(pr.first, 0, pr.second * 2, s);
    for (int k = 0; k < nk; ++k) {
        const size_t n = (size_t)nb[k] * naux;
        k_tc_pack_cce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(cc_dev[k], nb[k], naux, t->Kp_e, t->Mp_e, k, t->aeh,
                                                                  t->ael, flag);
        k_tc_pack_ccp<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(cc_dev[k], nb[k], naux, t->Kp_p, t->Mp_p, k, t->aph,
                                                                  t->apl, flag);
    }
    int e = tc_tmap3(&t->taeh, t->aeh, t->Kp_e, t->Mp_e, nk, TC_BM) | tc_tmap3(&t->tael, t->ael, t->Kp_e, t->Mp_e, nk, TC_BM) |
            tc_tmap3(&t->taph, t->aph, t->Kp_p, t->Mp_p, nk, TC_BM) | tc_tmap3(&t->tapl, t->apl, t->Kp_p, t->Mp_p, nk, TC_BM) |
            tc_tmap3(&t->tbeh, t->beh, t->Kp_e, t->NT, nk, t->NT) | tc_tmap3(&t->tbel, t->bel, t->Kp_e, t->NT, nk, t->NT) |
            tc_tmap3(&t->tbph, t->bph, t->Kp_p, t->NT, nk, t->NT) | tc_tmap3(&t->tbpl, t->bpl, t->Kp_p, t->NT, nk, t->NT);
    // the attribute is global per kernel: raise it to this plan's need, never lower it
    cudaError_t ce = cudaSuccess;
    switch (t->NT) {
#define RTD_TCO(n) \
    case n: ce = raise_smem((const void*)k_tc_opfwd<n>, (int)t->smem); break;
        RTD_TCO(16) RTD_TCO(32) RTD_TCO(48) RTD_TCO(64) RTD_TCO(96) RTD_TCO(128)
#undef RTD_TCO
    }
    if (e || ce != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        tc_cc_destroy(t);
        *why = "set-up of the tensor-core products with the auxiliary basis failed";
        return RTTDDFT_ERR_CUDA;
    }
    *out = t;
    return RTTDDFT_OK;
}

static void tcc_product(const TcCC* t, int proj, const KDev* kd, int nk, int* flag, cudaStream_t s) {
    TcOpParams p{};
    p.nk = nk;
    p.ns = t->ns;
    p.Dn = t->Dn;
    p.S = t->S;
    p.fmt = 1;
    p.kd = kd;
    p.flag = flag;
    if (proj) {
        p.ma = t->naux;
        p.kbps = t->kbps_p;
        p.splits = t->splits_p;
        p.atiles = t->tiles_p;
        p.R = t->Mp_p;
        p.k_nb = 1;
        p.rows_ng = 0;
        p.D = t->Dp;
    } else {
        p.kbps = t->nkb_e;
        p.splits = 1;
        p.atiles = t->tiles_e;
        p.R = t->Mp_e;
        p.nkb_fixed = t->nkb_e;
        p.rows_ng = 2;
        p.D = t->De;
    }
    dim3 g(p.atiles, p.splits, nk);
    const CUtensorMap &bh = proj ? t->tbph : t->tbeh, &bl = proj ? t->tbpl : t->tbel;
    const CUtensorMap &ah = proj ? t->taph : t->taeh, &al = proj ? t->tapl : t->tael;
    switch (t->NT) {
#define RTD_TCO(n) \
    case n: k_tc_opfwd<n><<<g, TCO_THREADS, t->smem, s>>>(bh, bl, ah, al, p); break;
        RTD_TCO(16) RTD_TCO(32) RTD_TCO(48) RTD_TCO(64) RTD_TCO(96) RTD_TCO(128)
#undef RTD_TCO
    }
}

// C = CC theta: pack theta, the product, the sums into K.C; returns the launches
int launch_tcc_expand(const TcCC* t, const StepArgs& a, cudaStream_t s) {
    k_tc_pack_cols<<<dim3((t->naux * t->ns + 255) / 256, 1, a.nk), 256, 0, s>>>(a.kd, 0, t->ns, t->naux, t->naux,
                                                                                t->Kp_e, t->NT, t->beh, t->bel, a.flag);
    tcc_product(t, 0, a.kd, a.nk, a.flag, s);
    TcCCRed r{0, t->ns, t->naux, t->Dn, t->Mp_e, 1, t->nkb_e, a.kd, t->De, nullptr};
    k_tc_ccred<<<dim3((t->maxnb + TC_RT - 1) / TC_RT, 1, a.nk), 256, 0, s>>>(r);
    return 3;
}
// theta~ partials = CC^H (S C) into part (one slice per k-point, k * naux * ns apart)
int launch_tcc_project(const TcCC* t, const StepArgs& a, zd* part, cudaStream_t s) {
    k_tc_pack_cols<<<dim3((t->maxnb * t->ns + 255) / 256, 1, a.nk), 256, 0, s>>>(a.kd, 1, t->ns, t->naux, t->maxnb,
                                                                                 t->Kp_p, t->NT, t->bph, t->bpl, a.flag);
    tcc_product(t, 1, a.kd, a.nk, a.flag, s);
    TcCCRed r{1, t->ns, t->naux, t->Dn, t->Mp_p, t->splits_p, t->kbps_p, a.kd, t->Dp, part};
    k_tc_ccred<<<dim3((t->naux + TC_RT - 1) / TC_RT, 1, a.nk), 256, 0, s>>>(r);
    return 3;
}

// ============================================================================
// The muffin-tin blocks of the operator (Eq. v_MT, with the momentum blocks of
// the current) as one batch of split-BF16 products on the matching-row
// pipeline: per (k, atom) W = G V with G the atom's 5m x m stack
// [h_eff; o; p_x; p_y; p_z] (h_eff = h + (A/c).p + |A|^2/2c^2 o + s dh, formed in
// FP64 each step) and V = [Q_alpha; C_lo,alpha] (m x N_s).  G is the left
// operand (K over the atom's m channels), V the right one; the FP32 products
// are converted into the FP64 W that the muffin-tin epilogue distributes.
// ============================================================================
struct TcMT {
    int nat = 0, nent = 0, maxm = 0, ns = 0, NT = 0, Dn = 0, Mp = 0, Kp = 0, nkb = 0, tiles = 0, S = 2;
    size_t smem = 0;
    unsigned short *ah = nullptr, *al = nullptr, *bh = nullptr, *bl = nullptr;
    float* D = nullptr;
    CUtensorMap tah, tal, tbh, tbl;
};

void tc_mt_destroy(TcMT* t) {
    if (!t) return;
    for (void* q : {(void*)t->ah, (void*)t->al, (void*)t->bh, (void*)t->bl, (void*)t->D}) cudaFree(q);
    delete t;
}

int tc_mt_create(TcMT** out, int nk, int nat, int maxm, int ns, int* flag, cudaStream_t s, std::string* why) {
    *out = nullptr;
    if (!get_encode()) {
        *why = "the driver has no tensor-map encoder";
        return RTTDDFT_ERR_UNSUPPORTED;
    }
    TcMT* t = new TcMT();
    t->nat = nat;
    t->nent = nk * nat;
    t->maxm = maxm;
    t->ns = ns;
    t->Dn = 2 * ns;
    for (int nt : TCO_NTS)
        if (nt >= t->Dn) {
            t->NT = nt;
            break;
        }
    if (!t->NT || t->NT > 128) {
        delete t;
        *why = "the tensor-core muffin-tin products take at most 64 states";
        return RTTDDFT_ERR_UNSUPPORTED;
    }
    int dev = 0, smax = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    t->nkb = (maxm + 31) / 32;
    t->Kp = t->nkb * TC_BK;
    t->tiles = (5 * maxm + TC_BM - 1) / TC_BM;
    t->Mp = t->tiles * TC_BM;
    const size_t stage = (size_t)2 * TC_BM * TC_BK * 2 + (size_t)2 * t->NT * TC_BK * 2;
    t->S = 4;
    while (t->S > 2 && 1024 + t->S * stage > (size_t)smax - 512) --t->S;
    t->smem = 1024 + t->S * stage;
    const size_t na = (size_t)nat * t->Mp * t->Kp, nb = (size_t)t->nent * t->NT * t->Kp;
    const size_t nd = (size_t)t->nent * t->Mp * t->Dn;
    if (cudaMalloc(&t->ah, na * 2) != cudaSuccess || cudaMalloc(&t->al, na * 2) != cudaSuccess ||
        cudaMalloc(&t->bh, nb * 2) != cudaSuccess || cudaMalloc(&t->bl, nb * 2) != cudaSuccess ||
        cudaMalloc(&t->D, nd * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        tc_mt_destroy(t);
        *why = "out of device memory for the tensor-core muffin-tin products";
        return RTTDDFT_ERR_OOM;
    }
    // padding rows and K columns stay zero: the packers write the atoms' own entries only
    for (auto pr : {std::make_pair((void*)t->ah, na), std::make_pair((void*)t->al, na),
                    std::make_pair((void*)t->bh, nb), std::make_pair((void*)t->bl, nb)})
        cudaMemsetAsync(pr.first, 0, pr.second * 2, s);
    int e = tc_tmap3(&t->tah, t->ah, t->Kp, t->Mp, nat, TC_BM) | tc_tmap3(&t->tal, t->al, t->Kp, t->Mp, nat, TC_BM) |
            tc_tmap3(&t->tbh, t->bh, t->Kp, t->NT, t->nent, t->NT) |
            tc_tmap3(&t->tbl, t->bl, t->Kp, t->NT, t->nent, t->NT);
    cudaError_t ce = cudaSuccess;
    switch (t->NT) {
#define RTD_TCO(n) \
    case n: ce = raise_smem((const void*)k_tc_opfwd<n>, (int)t->smem); break;
        RTD_TCO(16) RTD_TCO(32) RTD_TCO(48) RTD_TCO(64) RTD_TCO(96) RTD_TCO(128)
#undef RTD_TCO
    }
    (void)flag;
    if (e || ce != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        tc_mt_destroy(t);
        *why = "set-up of the tensor-core muffin-tin products failed";
        return RTTDDFT_ERR_CUDA;
    }
    *out = t;
    return RTTDDFT_OK;
}

// left operand of a step: per atom the rows of [h_eff; o; p_x; p_y; p_z] with K
// over the columns j of the m x m blocks (row r of the stack: [Re G(r, .) | Im
// G(r, .)] per K block of 32), one thread per (i, j) of the atom's blocks
__global__ void k_tc_mt_pack_a(StepArgs a, int Mp, int Kp, unsigned short* __restrict__ ah,
                               unsigned short* __restrict__ al) {
    const AtomTab& at = *a.at;
    const int atom = blockIdx.y;
    if (atom >= at.n) return;
    const int m = at.m[atom];
    const size_t mm = (size_t)m * m, bo = at.boff[atom];
    const DevState* st = a.st;
    const double fx = st->cur_a[0] * a.inv_c, fy = st->cur_a[1] * a.inv_c, fz = st->cur_a[2] * a.inv_c;
    const double fa = st->cur_aa, sdv = st->cur_s;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < mm; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % m), j = (int)(e / m);
        const zd hv = a.h[bo + e], ov = a.o[bo + e];
        const zd px = a.p[3 * bo + e], py = a.p[3 * bo + mm + e], pz = a.p[3 * bo + 2 * mm + e];
        zd he = zmk(hv.x + fx * px.x + fy * py.x + fz * pz.x + fa * ov.x,
                    hv.y + fx * px.y + fy * py.y + fz * pz.y + fa * ov.y);
        if (a.dh && sdv != 0.0) {
            const zd d = a.dh[bo + e];
            he.x += sdv * d.x;
            he.y += sdv * d.y;
        }
        const zd blk[5] = {he, ov, px, py, pz};
        const size_t col = (size_t)(j >> 5) * 64 + (j & 31);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const size_t row = ((size_t)atom * Mp + q * m + i) * Kp + col;
            put16(blk[q].x, 1, 1.0, ah, al, row, a.flag);
            put16(blk[q].y, 1, 1.0, ah, al, row + 32, a.flag);
        }
    }
}
// right operand of a step from the gathered V = [Q; C_lo] of every (k, atom) of
// the call: rows c < ns hold [Re V | -Im V], rows ns + c [Im V | Re V] over K = i
__global__ void k_tc_mt_pack_b(StepArgs a, int NT, int Kp, unsigned short* __restrict__ bh,
                               unsigned short* __restrict__ bl) {
    const AtomTab& at = *a.at;
    const int atom = blockIdx.y, k = blockIdx.z;
    if (atom >= at.n) return;
    const int m = at.m[atom], ns = a.ns;
    const size_t ent = (size_t)(a.kofs + k) * at.n + atom;
    const zd* V = a.mtv + ent * a.mtv_stride;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * ns; e += gridDim.x * blockDim.x) {
        const int i = e % m, c = e / m;
        const zd x = V[e];
        const size_t kc = (size_t)(i >> 5) * 64 + (i & 31);
        const size_t re_row = (ent * NT + c) * Kp + kc, im_row = (ent * NT + ns + c) * Kp + kc;
        put16(x.x, 1, 1.0, bh, bl, re_row, a.flag);
        put16(-x.y, 1, 1.0, bh, bl, re_row + 32, a.flag);
        put16(x.y, 1, 1.0, bh, bl, im_row, a.flag);
        put16(x.x, 1, 1.0, bh, bl, im_row + 32, a.flag);
    }
}
// W (FP64, 5m x N_s per (k, atom), column-major) from the FP32 products
// D[z][row][Re c | Im c] of the call's entries z = k n_atoms + atom
__global__ void k_tc_mt_w(StepArgs a, const float* __restrict__ D, int Mp, int Dn) {
    const AtomTab& at = *a.at;
    const int atom = blockIdx.y, k = blockIdx.z;
    if (atom >= at.n) return;
    const int m5 = 5 * at.m[atom], ns = a.ns;
    const size_t z = (size_t)k * at.n + atom;
    const size_t ent = (size_t)(a.kofs + k) * at.n + atom;
    zd* W = a.mtw + ent * a.mtw_stride;
    const float* d = D + z * Mp * Dn;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m5 * ns; e += gridDim.x * blockDim.x) {
        const int r = e % m5, c = e / m5;
        W[e] = zmk((double)d[(size_t)r * Dn + c], (double)d[(size_t)r * Dn + ns + c]);
    }
}

int launch_tc_mt(const TcMT* t, const StepArgs& a, cudaStream_t s) {
    const int nat = t->nat;
    k_tc_mt_pack_a<<<dim3(64, nat), 256, 0, s>>>(a, t->Mp, t->Kp, t->ah, t->al);
    k_tc_mt_pack_b<<<dim3((t->maxm * t->ns + 255) / 256, nat, a.nk), 256, 0, s>>>(a, t->NT, t->Kp, t->bh, t->bl);
    TcOpParams p{};
    p.nk = a.nk * nat;
    p.ns = t->ns;
    p.ma = t->Mp;
    p.Dn = t->Dn;
    p.kbps = t->nkb;
    p.splits = 1;
    p.atiles = t->tiles;
    p.R = t->Mp;
    p.S = t->S;
    p.nkb_fixed = t->nkb;
    p.rows_ng = 0;
    p.fmt = 1;
    p.a_zmod = nat;
    p.bz0 = a.kofs * nat;
    p.kd = a.kd;
    p.D = t->D;
    p.flag = a.flag;
    const dim3 g(t->tiles, 1, a.nk * nat);
    switch (t->NT) {
#define RTD_TCO(n) \
    case n: k_tc_opfwd<n><<<g, TCO_THREADS, t->smem, s>>>(t->tbh, t->tbl, t->tah, t->tal, p); break;
        RTD_TCO(16) RTD_TCO(32) RTD_TCO(48) RTD_TCO(64) RTD_TCO(96) RTD_TCO(128)
#undef RTD_TCO
    }
    k_tc_mt_w<<<dim3((5 * t->maxm * t->ns + 255) / 256, nat, a.nk), 256, 0, s>>>(a, t->D, t->Mp, t->Dn);
    return 4;
}
