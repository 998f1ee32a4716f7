// Batched complex contractions used by the step and its set-up.
//
// On GB300 the FP64 pipe delivers a few DFMA per clock per SM, so an FP64
// complex contraction is bound by its multiply-add count even at two
// right-hand columns; these kernels keep every DFMA useful and spread the
// work over all SMs (split-K where the output is small).  The FP32-storage
// variants stream half the bytes and run on the FFMA pipe.
#include <algorithm>

#include "rtd.h"

// ---------------------------------------------------------------- NN
// C[m, n] (+)= sum_k A[m, k] B[k, n].  A block has 64 output rows and four
// k-groups (256 threads); a K-chunk of B is staged in shared memory and the
// four groups' partial sums are combined in shared memory, so a column of A
// is read once and coalesced.  NT columns per pass; split-K over blockIdx.y.
template <typename TA, typename TC, int NT>
__global__ void __launch_bounds__(256) k_gemm_nn(const GemmDesc* __restrict__ descs, int N,
                                                 int kchunk, zd* __restrict__ part, int beta_add,
                                                 const double* __restrict__ dscale, int ncg) {
    const GemmDesc d = descs[blockIdx.z];
    // blockIdx.x = row tile + mtiles x column group: the column chunks of NT are
    // spread over ncg groups of blocks
    const int mtiles = (gridDim.x + ncg - 1) / ncg;
    const int mt = blockIdx.x % mtiles, cg = blockIdx.x / mtiles;
    const int m0 = mt * 64;
    const int k0 = blockIdx.y * kchunk;
    if (m0 >= d.M || k0 >= d.K) return;
    const int k1 = min(d.K, k0 + kchunk);
    const int r = threadIdx.x & 63, grp = threadIdx.x >> 6;
    const int m = m0 + r;
    const bool act = m < d.M;
    const TA* __restrict__ A = (const TA*)d.A;
    __shared__ TC bs[64][NT];
    __shared__ TC red[3][64][NT];
    for (int n0 = cg * NT; n0 < N; n0 += NT * ncg) {
        TC acc[NT];
#pragma unroll
        for (int j = 0; j < NT; ++j) acc[j] = Cx<TC>::zero();
        for (int kb = k0; kb < k1; kb += 64) {
            __syncthreads();
            for (int e = threadIdx.x; e < 64 * NT; e += 256) {
                const int kk = e & 63, j = e >> 6;
                const int kg = kb + kk, n = n0 + j;
                bs[kk][j] = (kg < k1 && n < N) ? Cx<TC>::from(d.B[kg + (size_t)n * d.ldb]) : Cx<TC>::zero();
            }
            __syncthreads();
            if (act) {
                const int kend = min(64, k1 - kb);
                const TA* ap = A + m + (size_t)kb * d.lda;
                for (int kk = grp; kk < kend; kk += 4) {
                    const TC a = Cx<TC>::from(ap[(size_t)kk * d.lda]);
#pragma unroll
                    for (int j = 0; j < NT; ++j) Cx<TC>::fma(acc[j], a, bs[kk][j]);
                }
            }
        }
        if (grp > 0) {
#pragma unroll
            for (int j = 0; j < NT; ++j) red[grp - 1][r][j] = acc[j];
        }
        __syncthreads();
        if (grp == 0 && act) {
            const double sc = dscale ? *dscale : 1.0;
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const int n = n0 + j;
                if (n >= N) break;
                zd v = zadd(zadd(Cx<TC>::todbl(acc[j]), Cx<TC>::todbl(red[0][r][j])),
                            zadd(Cx<TC>::todbl(red[1][r][j]), Cx<TC>::todbl(red[2][r][j])));
                v = zscale(v, sc);
                if (part) {
                    part[d.part_off + ((size_t)blockIdx.y * N + n) * d.M + m] = v;
                } else {
                    zd* c = d.C + m + (size_t)n * d.ldc;
                    *c = beta_add ? zadd(*c, v) : v;
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- CN
// C[m, n] (+)= sum_k conj(A[k, m]) B[k, n].  Eight warps, each owning RPW
// output rows; lanes stride over k (column m of A is contiguous) and a
// K-chunk of B staged in shared memory serves the block's 8 RPW rows.
template <typename TA, typename TC, int NT, int RPW>
__global__ void __launch_bounds__(256) k_gemm_cn(const GemmDesc* __restrict__ descs, int N,
                                                 int kchunk, zd* __restrict__ part, int beta_add,
                                                 const double* __restrict__ dscale, int ncg) {
    const GemmDesc d = descs[blockIdx.z];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mtiles = (gridDim.x + ncg - 1) / ncg;
    const int cg = blockIdx.x / mtiles;
    const int mb = (blockIdx.x % mtiles) * 8 * RPW;
    const int k0 = blockIdx.y * kchunk;
    if (mb >= d.M || k0 >= d.K) return;
    const int k1 = min(d.K, k0 + kchunk);
    const int m0 = mb + warp * RPW;
    __shared__ TC bs[128][NT];
    for (int n0 = cg * NT; n0 < N; n0 += NT * ncg) {
        TC acc[RPW][NT];
#pragma unroll
        for (int q = 0; q < RPW; ++q)
#pragma unroll
            for (int j = 0; j < NT; ++j) acc[q][j] = Cx<TC>::zero();
        for (int kb = k0; kb < k1; kb += 128) {
            __syncthreads();
            for (int e = threadIdx.x; e < 128 * NT; e += 256) {
                const int kk = e & 127, j = e >> 7;
                const int kg = kb + kk, n = n0 + j;
                bs[kk][j] = (kg < k1 && n < N) ? Cx<TC>::from(d.B[kg + (size_t)n * d.ldb]) : Cx<TC>::zero();
            }
            __syncthreads();
            const int kend = min(128, k1 - kb);
            if (kend == 128 && m0 + RPW <= d.M) {
                // full chunk: issue all 4 RPW loads before the multiply-adds
                TA av[RPW][4];
#pragma unroll
                for (int q = 0; q < RPW; ++q) {
                    const TA* ap = (const TA*)d.A + (size_t)(m0 + q) * d.lda + kb + lane;
#pragma unroll
                    for (int u = 0; u < 4; ++u) av[q][u] = ap[32 * u];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int q = 0; q < RPW; ++q) {
                        const TC a = Cx<TC>::from(av[q][u]);
#pragma unroll
                        for (int j = 0; j < NT; ++j) Cx<TC>::fmac(acc[q][j], a, bs[lane + 32 * u][j]);
                    }
            } else {
#pragma unroll
                for (int q = 0; q < RPW; ++q) {
                    const int m = m0 + q;
                    if (m >= d.M) break;
                    const TA* ap = (const TA*)d.A + (size_t)m * d.lda + kb;
                    for (int kk = lane; kk < kend; kk += 32) {
                        const TC a = Cx<TC>::from(ap[kk]);
#pragma unroll
                        for (int j = 0; j < NT; ++j) Cx<TC>::fmac(acc[q][j], a, bs[kk][j]);
                    }
                }
            }
        }
        const double sc = dscale ? *dscale : 1.0;
#pragma unroll
        for (int q = 0; q < RPW; ++q) {
            const int m = m0 + q;
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const zd s = zscale(warp_zsum(Cx<TC>::todbl(acc[q][j])), sc);
                const int n = n0 + j;
                if (lane == j && n < N && m < d.M) {
                    if (part) {
                        part[d.part_off + ((size_t)blockIdx.y * N + n) * d.M + m] = s;
                    } else {
                        zd* c = d.C + m + (size_t)n * d.ldc;
                        *c = beta_add ? zadd(*c, s) : s;
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------- FP32 streaming forms
// The same products with A in FP32 (FP32 and split-BF16 precision forms),
// written for streaming A at full memory bandwidth: every thread issues all
// of its loads of A for the block's K range before it waits on anything,
// the block's slice of B is staged once in shared memory (as FP32) while
// those loads are in flight, and there is no synchronisation inside the K
// loop.  Sums are FP32 within a block, FP64 across split-K slices.

// CN: C[m, n] (+)= sum_k conj(A[k, m]) B[k, n]; warp = RPW rows, lanes over k
template <int NT, int RPW, int KC>
__global__ void __launch_bounds__(256) k_gemm_cn32(const GemmDesc* __restrict__ descs, int N, int kchunk,
                                                   zd* __restrict__ part, int beta_add,
                                                   const double* __restrict__ dscale,
                                                   unsigned* __restrict__ tile_cnt) {
    constexpr int U = KC / 32;  // loads of A per lane and row
    __shared__ zf bs[KC][NT];
    __shared__ float red[8][2 * RPW * NT];
    const GemmDesc d = descs[blockIdx.z];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mb = blockIdx.x * 8 * RPW;
    const int k0 = blockIdx.y * kchunk;  // kchunk <= KC
    if (mb >= d.M || k0 >= d.K) return;
    const int kn = min(kchunk, d.K - k0);
    const int m0 = mb + warp * RPW;
    const zf* __restrict__ A = (const zf*)d.A;
    for (int n0 = 0; n0 < N; n0 += NT) {
        zf av[RPW][U];
#pragma unroll
        for (int q = 0; q < RPW; ++q)
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int kk = lane + 32 * u;
                av[q][u] = (m0 + q < d.M && kk < kn) ? A[(size_t)(m0 + q) * d.lda + k0 + kk] : make_float2(0.f, 0.f);
            }
        __syncthreads();
        for (int e = threadIdx.x; e < KC * NT; e += 256) {
            const int kk = e / NT, j = e % NT;
            bs[kk][j] = (kk < kn && n0 + j < N) ? tof(d.B[k0 + kk + (size_t)(n0 + j) * d.ldb]) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        zf acc[RPW][NT];
#pragma unroll
        for (int q = 0; q < RPW; ++q)
#pragma unroll
            for (int j = 0; j < NT; ++j) acc[q][j] = make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int kk = lane + 32 * u;
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const zf b = bs[kk][j];
#pragma unroll
                for (int q = 0; q < RPW; ++q) cfmac(acc[q][j], av[q][u], b);
            }
        }
        float v[2 * RPW * NT];
#pragma unroll
        for (int q = 0; q < RPW; ++q)
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                v[2 * (q * NT + j)] = acc[q][j].x;
                v[2 * (q * NT + j) + 1] = acc[q][j].y;
            }
        warp_sum_store<float, 2 * RPW * NT>(v, lane, red[warp]);
        __syncwarp();
        const double sc = dscale ? *dscale : 1.0;
        for (int e = lane; e < RPW * NT; e += 32) {
            const int q = e / NT, j = e % NT;
            const int m = m0 + q, n = n0 + j;
            if (m >= d.M || n >= N) continue;
            const zd val = zscale(zmk((double)red[warp][2 * e], (double)red[warp][2 * e + 1]), sc);
            if (part) {
                part[d.part_off + ((size_t)blockIdx.y * N + n) * d.M + m] = val;
            } else {
                zd* c = d.C + m + (size_t)n * d.ldc;
                *c = beta_add ? zadd(*c, val) : val;
            }
        }
    }
    if (!part || !tile_cnt) return;
    // the last K slice of this row tile to finish sums the slices in slice
    // order (the same sums as k_split_reduce, whichever block is last)
    __shared__ unsigned last;
    __threadfence();
    __syncthreads();
    const int nsp = (d.K + kchunk - 1) / kchunk;
    if (threadIdx.x == 0) {
        unsigned* c = tile_cnt + (size_t)blockIdx.z * gridDim.x + blockIdx.x;
        last = (atomicAdd(c, 1u) == (unsigned)(nsp - 1)) ? 1u : 0u;
        if (last) *c = 0u;  // ready for the next launch
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int rows = 8 * RPW;
    const size_t st = (size_t)N * d.M;
    for (int e = threadIdx.x; e < rows * N; e += 256) {
        const int m = mb + e % rows, n = e / rows;
        if (m >= d.M) continue;
        const zd* p = part + d.part_off + (size_t)n * d.M + m;
        zd sum = zmk(0.0, 0.0);
        int sp = 0;
        for (; sp + 8 <= nsp; sp += 8) {
            zd t[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) t[u] = __ldcg(p + (size_t)(sp + u) * st);
#pragma unroll
            for (int u = 0; u < 8; ++u) sum = zadd(sum, t[u]);
        }
        for (; sp < nsp; ++sp) sum = zadd(sum, __ldcg(p + (size_t)sp * st));
        zd* c = d.C + m + (size_t)n * d.ldc;
        *c = beta_add ? zadd(*c, sum) : sum;
    }
}

// NN: C[m, n] (+)= sum_k A[m, k] B[k, n]; thread = row, four k-groups per
// block of 64 rows, the block's K slice (at most KC) of B in shared memory
template <int NT, int KC>
__global__ void __launch_bounds__(256) k_gemm_nn32(const GemmDesc* __restrict__ descs, int N, int kchunk,
                                                   zd* __restrict__ part, int beta_add,
                                                   const double* __restrict__ dscale) {
    constexpr int U = 8;
    __shared__ zf bs[KC][NT];
    __shared__ zf redc[3][64][NT];
    const GemmDesc d = descs[blockIdx.z];
    const int m0 = blockIdx.x * 64;
    const int k0 = blockIdx.y * kchunk;
    if (m0 >= d.M || k0 >= d.K) return;
    const int kn = min(kchunk, d.K - k0);
    const int r = threadIdx.x & 63, grp = threadIdx.x >> 6;
    const int m = m0 + r;
    const bool act = m < d.M;
    const zf* __restrict__ A = (const zf*)d.A + m;
    for (int n0 = 0; n0 < N; n0 += NT) {
        // the first loads of A go out before the slice of B is staged; two
        // register buffers alternate so that the next chunk is always in flight
        zf a0[U], a1[U];
        auto load = [&](zf* dst, int kb) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int kk = kb + 4 * u;
                dst[u] = (act && kk < kn) ? A[(size_t)(k0 + kk) * d.lda] : make_float2(0.f, 0.f);
            }
        };
        zf acc[NT];
#pragma unroll
        for (int j = 0; j < NT; ++j) acc[j] = make_float2(0.f, 0.f);
        auto fma_chunk = [&](const zf* av, int kb) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int kk = kb + 4 * u;
                if (kk < kn) {
#pragma unroll
                    for (int j = 0; j < NT; ++j) cfma(acc[j], av[u], bs[kk][j]);
                }
            }
        };
        load(a0, grp);
        __syncthreads();
        for (int e = threadIdx.x; e < kn * NT; e += 256) {
            const int kk = e / NT, j = e % NT;
            bs[kk][j] = (n0 + j < N) ? tof(d.B[k0 + kk + (size_t)(n0 + j) * d.ldb]) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int kb = grp; kb < kn; kb += 8 * U) {
            if (kb + 4 * U < kn) load(a1, kb + 4 * U);
            fma_chunk(a0, kb);
            if (kb + 4 * U >= kn) break;
            if (kb + 8 * U < kn) load(a0, kb + 8 * U);
            fma_chunk(a1, kb + 4 * U);
        }
        if (grp > 0) {
#pragma unroll
            for (int j = 0; j < NT; ++j) redc[grp - 1][r][j] = acc[j];
        }
        __syncthreads();
        if (grp == 0 && act) {
            const double sc = dscale ? *dscale : 1.0;
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const int n = n0 + j;
                if (n >= N) break;
                zd v = zadd(zadd(tod(acc[j]), tod(redc[0][r][j])), zadd(tod(redc[1][r][j]), tod(redc[2][r][j])));
                v = zscale(v, sc);
                if (part) {
                    part[d.part_off + ((size_t)blockIdx.y * N + n) * d.M + m] = v;
                } else {
                    zd* c = d.C + m + (size_t)n * d.ldc;
                    *c = beta_add ? zadd(*c, v) : v;
                }
            }
        }
    }
}

__global__ void k_split_reduce(const GemmDesc* __restrict__ descs, int N, int kchunk,
                               const zd* __restrict__ part, int beta_add) {
    const GemmDesc d = descs[blockIdx.z];
    const int idx = blockIdx.x * 256 + threadIdx.x;
    if (idx >= d.M * N) return;
    const int m = idx % d.M, n = idx / d.M;
    const int nsp = (d.K + kchunk - 1) / kchunk;
    zd s = zmk(0.0, 0.0);
    const zd* p = part + d.part_off + (size_t)n * d.M + m;
    const size_t st = (size_t)N * d.M;
    int sp = 0;
    for (; sp + 8 <= nsp; sp += 8) {
        zd t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) t[u] = p[(size_t)(sp + u) * st];
#pragma unroll
        for (int u = 0; u < 8; ++u) s = zadd(s, t[u]);
    }
    for (; sp < nsp; ++sp) s = zadd(s, p[(size_t)sp * st]);
    zd* c = d.C + m + (size_t)n * d.ldc;
    *c = beta_add ? zadd(*c, s) : s;
}

// column groups for the generic kernels: enough blocks to cover about two per
// SM, at most one group per column chunk
static int column_groups(int blocks, int chunks) {
    int g = (2 * 152 + blocks - 1) / std::max(blocks, 1);
    return std::max(1, std::min(g, chunks));
}

template <typename TA, typename TC>
static void gemm_nn_t(const GemmDesc* d, int nb, int maxM, int maxK, int N, int kchunk, zd* part,
                      int beta_add, const double* ds, cudaStream_t s) {
    if (nb <= 0 || maxM <= 0 || maxK <= 0 || N <= 0) return;
    if (kchunk <= 0) kchunk = maxK;
    const int NTb = N <= 2 ? 2 : (N <= 4 ? 4 : 8);
    const int mt = (maxM + 63) / 64, ks = (maxK + kchunk - 1) / kchunk;
    const int ncg = column_groups(mt * ks * nb, (N + NTb - 1) / NTb);
    dim3 grid(mt * ncg, ks, nb);
    if (N <= 2)
        k_gemm_nn<TA, TC, 2><<<grid, 256, 0, s>>>(d, N, kchunk, part, beta_add, ds, ncg);
    else if (N <= 4)
        k_gemm_nn<TA, TC, 4><<<grid, 256, 0, s>>>(d, N, kchunk, part, beta_add, ds, ncg);
    else
        k_gemm_nn<TA, TC, 8><<<grid, 256, 0, s>>>(d, N, kchunk, part, beta_add, ds, ncg);
}
template <typename TA, typename TC>
static void gemm_cn_t(const GemmDesc* d, int nb, int maxM, int maxK, int N, int kchunk, zd* part,
                      int beta_add, const double* ds, cudaStream_t s) {
    if (nb <= 0 || maxM <= 0 || maxK <= 0 || N <= 0) return;
    if (kchunk <= 0) kchunk = maxK;
    const int ks = (maxK + kchunk - 1) / kchunk;
    if (N <= 2) {
        dim3 grid((maxM + 31) / 32, ks, nb);
        k_gemm_cn<TA, TC, 2, 4><<<grid, 256, 0, s>>>(d, N, kchunk, part, beta_add, ds, 1);
    } else if (N <= 4) {
        dim3 grid((maxM + 15) / 16, ks, nb);
        k_gemm_cn<TA, TC, 4, 2><<<grid, 256, 0, s>>>(d, N, kchunk, part, beta_add, ds, 1);
    } else {
        const int mt = (maxM + 7) / 8;
        const int ncg = column_groups(mt * ks * nb, (N + 7) / 8);
        dim3 grid(mt * ncg, ks, nb);
        k_gemm_cn<TA, TC, 8, 1><<<grid, 256, 0, s>>>(d, N, kchunk, part, beta_add, ds, ncg);
    }
}

// ---------------------------------------------------------------- FP32 tiles for many columns
// C[m, n] (+)= sum_k op(A)[m, k] B[k, n] with op(A) = A (CN = false, A is
// M x K) or A^H (CN = true, A is K x M), A in FP32, B read as FP64 and
// rounded to FP32 where it is staged.  A block owns a 64 x 64 tile of C and
// walks its K slice in steps of 16: both operand tiles sit in shared memory
// and every thread keeps 4 x 4 complex accumulators in registers (rows
// tx + 16 i, columns ty + 16 j), so each staged value feeds four products.
// The next step's operands are loaded into registers while the current
// step's products run.  FP32 sums within a K slice, FP64 across slices.
#define ZT_BM 64
#define ZT_BN 64
#define ZT_BK 16
template <bool CN>
__global__ void __launch_bounds__(256) k_zgemm_t32(const GemmDesc* __restrict__ descs, int N, int kchunk,
                                                   zd* __restrict__ part, int beta_add,
                                                   const double* __restrict__ dscale) {
    __shared__ zf As[2][ZT_BK][ZT_BM];
    __shared__ zf Bs[2][ZT_BK][ZT_BN];
    const GemmDesc d = descs[blockIdx.z];
    const int ntn = (N + ZT_BN - 1) / ZT_BN;
    const int m0 = (blockIdx.x / ntn) * ZT_BM, n0 = (blockIdx.x % ntn) * ZT_BN;
    const int k0 = blockIdx.y * kchunk;
    if (m0 >= d.M || k0 >= d.K) return;
    const int k1 = min(d.K, k0 + kchunk);
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const zf* __restrict__ A = (const zf*)d.A;
    const zd* __restrict__ B = d.B;
    zf ra[4], rb[4];
    // staging loads of one K step (kb): four A and four B values per thread
    auto fetch = [&](int kb) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (CN) {
                // conj(A[k, m]): k = kb + (t & 15) (contiguous), m = m0 + (t >> 4) + 16 i
                const int k = kb + tx, m = m0 + ty + 16 * i;
                ra[i] = (k < k1 && m < d.M) ? A[(size_t)m * d.lda + k] : make_float2(0.f, 0.f);
            } else {
                // A[m, k]: m = m0 + (t & 63) (contiguous), k = kb + (t >> 6) + 4 i
                const int m = m0 + (t & 63), k = kb + (t >> 6) + 4 * i;
                ra[i] = (k < k1 && m < d.M) ? A[m + (size_t)k * d.lda] : make_float2(0.f, 0.f);
            }
            const int k = kb + tx, n = n0 + ty + 16 * i;
            rb[i] = (k < k1 && n < N) ? tof(B[k + (size_t)n * d.ldb]) : make_float2(0.f, 0.f);
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (CN) As[buf][tx][ty + 16 * i] = make_float2(ra[i].x, -ra[i].y);
            else As[buf][(t >> 6) + 4 * i][t & 63] = ra[i];
            Bs[buf][tx][ty + 16 * i] = rb[i];
        }
    };
    zf acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    fetch(k0);
    stash(0);
    __syncthreads();
    int buf = 0;
    for (int kb = k0; kb < k1; kb += ZT_BK) {
        const bool more = kb + ZT_BK < k1;
        if (more) fetch(kb + ZT_BK);
#pragma unroll
        for (int kk = 0; kk < ZT_BK; ++kk) {
            zf a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[buf][kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[buf][kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
        }
        if (more) {
            stash(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
    const double sc = dscale ? *dscale : 1.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + tx + 16 * i;
        if (m >= d.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + ty + 16 * j;
            if (n >= N) continue;
            const zd v = zscale(tod(acc[i][j]), sc);
            if (part) {
                part[d.part_off + ((size_t)blockIdx.y * N + n) * d.M + m] = v;
            } else {
                zd* c = d.C + m + (size_t)n * d.ldc;
                *c = beta_add ? zadd(*c, v) : v;
            }
        }
    }
}

// largest K slice of a block in the FP32 streaming kernels
#define GEMM32_KC 256
void launch_gemm_nn(const GemmDesc* d, int nb, int maxM, int maxK, int N, int kchunk, zd* part,
                    int beta_add, bool a_fp32, const double* ds, cudaStream_t s) {
    if (a_fp32 && N >= ZT_MIN_N && nb > 0 && maxM > 0 && maxK > 0) {
        const int kc = kchunk > 0 ? kchunk : maxK;
        dim3 grid(((maxM + ZT_BM - 1) / ZT_BM) * ((N + ZT_BN - 1) / ZT_BN), (maxK + kc - 1) / kc, nb);
        k_zgemm_t32<false><<<grid, 256, 0, s>>>(d, N, kc, part, beta_add, ds);
        return;
    }
    if (a_fp32 && nb > 0 && maxM > 0 && maxK > 0 && N > 0 && (kchunk > 0 ? kchunk : maxK) <= GEMM32_KC) {
        const int kc = kchunk > 0 ? kchunk : maxK;
        dim3 grid((maxM + 63) / 64, (maxK + kc - 1) / kc, nb);
        if (N <= 2) k_gemm_nn32<2, GEMM32_KC><<<grid, 256, 0, s>>>(d, N, kc, part, beta_add, ds);
        else if (N <= 4) k_gemm_nn32<4, GEMM32_KC><<<grid, 256, 0, s>>>(d, N, kc, part, beta_add, ds);
        else k_gemm_nn32<8, GEMM32_KC><<<grid, 256, 0, s>>>(d, N, kc, part, beta_add, ds);
        return;
    }
    if (a_fp32) gemm_nn_t<zf, zf>(d, nb, maxM, maxK, N, kchunk, part, beta_add, ds, s);
    else gemm_nn_t<zd, zd>(d, nb, maxM, maxK, N, kchunk, part, beta_add, ds, s);
}
bool launch_gemm_cn(const GemmDesc* d, int nb, int maxM, int maxK, int N, int kchunk, zd* part,
                    int beta_add, bool a_fp32, const double* ds, cudaStream_t s, unsigned* tile_cnt) {
    if (a_fp32 && N >= ZT_MIN_N && nb > 0 && maxM > 0 && maxK > 0) {
        const int kc = kchunk > 0 ? kchunk : maxK;
        dim3 grid(((maxM + ZT_BM - 1) / ZT_BM) * ((N + ZT_BN - 1) / ZT_BN), (maxK + kc - 1) / kc, nb);
        k_zgemm_t32<true><<<grid, 256, 0, s>>>(d, N, kc, part, beta_add, ds);
        return false;
    }
    if (a_fp32 && nb > 0 && maxM > 0 && maxK > 0 && N > 0 && (kchunk > 0 ? kchunk : maxK) <= GEMM32_KC) {
        const int kc = kchunk > 0 ? kchunk : maxK;
        unsigned* tc = part ? tile_cnt : nullptr;
        if (N <= 2) {
            dim3 grid((maxM + 31) / 32, (maxK + kc - 1) / kc, nb);
            k_gemm_cn32<2, 4, GEMM32_KC><<<grid, 256, 0, s>>>(d, N, kc, part, beta_add, ds, tc);
        } else if (N <= 4) {
            dim3 grid((maxM + 15) / 16, (maxK + kc - 1) / kc, nb);
            k_gemm_cn32<4, 2, GEMM32_KC><<<grid, 256, 0, s>>>(d, N, kc, part, beta_add, ds, tc);
        } else {
            dim3 grid((maxM + 7) / 8, (maxK + kc - 1) / kc, nb);
            k_gemm_cn32<8, 1, GEMM32_KC><<<grid, 256, 0, s>>>(d, N, kc, part, beta_add, ds, tc);
        }
        return tc != nullptr;
    }
    if (a_fp32) gemm_cn_t<zf, zf>(d, nb, maxM, maxK, N, kchunk, part, beta_add, ds, s);
    else gemm_cn_t<zd, zd>(d, nb, maxM, maxK, N, kchunk, part, beta_add, ds, s);
    return false;
}
void launch_split_reduce(const GemmDesc* d, int nb, int maxM, int N, int kchunk, const zd* part,
                         int beta_add, cudaStream_t s) {
    if (nb <= 0 || maxM <= 0 || N <= 0) return;
    dim3 grid((maxM * N + 255) / 256, 1, nb);
    k_split_reduce<<<grid, 256, 0, s>>>(d, N, kchunk, part, beta_add);
}

// ---------------------------------------------------------------- Toeplitz
// Eq. v_interstitial as an operator: Y[G, n] (+)= sum_G' V~_{G-G'} X[G', n]
// (+ d_G X[G, n]).  The integer difference G - G' maps to a table offset
// glin(G) - glin(G') + center because the table box is dense.
template <int NT>
__global__ void __launch_bounds__(256) k_toeplitz(const KDev* __restrict__ kd, const ToepDesc* __restrict__ td,
                                                  int N, const zd* __restrict__ tab, int center,
                                                  int beta_add, int dmode,
                                                  const double* __restrict__ dscale) {
    const int k = blockIdx.z;
    const int ng = kd[k].ng;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * 8 + warp;
    if (g >= ng) return;
    const ToepDesc t = td[k];
    const int* __restrict__ glin = kd[k].glin;
    const int base = glin[g] + center;
    double dg = 0.0;
    if (dmode == 1) {
        const double* q = kd[k].gk + 3 * (size_t)g;
        dg = 0.5 * (q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    } else if (dmode >= 2 && dmode <= 4) {
        dg = kd[k].gk[3 * (size_t)g + (dmode - 2)];
    } else if (dmode == 5) {
        dg = 1.0;
    }
    for (int n0 = 0; n0 < N; n0 += NT) {
        zd acc[NT];
#pragma unroll
        for (int j = 0; j < NT; ++j) acc[j] = zmk(0.0, 0.0);
        if (tab) {
            for (int gp = lane; gp < ng; gp += 32) {
                const zd v = tab[base - glin[gp]];
#pragma unroll
                for (int j = 0; j < NT; ++j)
                    if (n0 + j < N) zfma(acc[j], v, t.X[gp + (size_t)(n0 + j) * t.ldx]);
            }
        }
        const double sc = dscale ? *dscale : 1.0;
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            zd s = zscale(warp_zsum(acc[j]), sc);
            const int n = n0 + j;
            if (lane == j && n < N) {
                if (dmode) s = zadd(s, zscale(t.X[g + (size_t)n * t.ldx], dg));
                zd* y = t.Y + g + (size_t)n * t.ldy;
                *y = beta_add ? zadd(*y, s) : s;
            }
        }
    }
}

void launch_toeplitz(const KDev* kd, const ToepDesc* td, int nk, int maxng, int N, const zd* tab,
                     int center, int beta_add, int dmode, const double* dscale, cudaStream_t s) {
    if (nk <= 0 || maxng <= 0 || N <= 0) return;
    dim3 grid((maxng + 7) / 8, 1, nk);
    k_toeplitz<8><<<grid, 256, 0, s>>>(kd, td, N, tab, center, beta_add, dmode, dscale);
}

__global__ void k_zero(zd* p, size_t n) {
    size_t i = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (i < n) p[i] = zmk(0.0, 0.0);
}
void launch_zero(zd* p, size_t n, cudaStream_t s) {
    if (n == 0) return;
    k_zero<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n);
}

// C[r, c] = B[r, c] for r < M, c < K (batched strided copy; GemmDesc fields B, C, M, K, ldb, ldc)
__global__ void k_copy_rows(const GemmDesc* __restrict__ descs, int ncol) {
    const GemmDesc d = descs[blockIdx.z];
    const int e = blockIdx.x * 256 + threadIdx.x;
    if (e >= d.M * ncol) return;
    const int r = e % d.M, c = e / d.M;
    d.C[r + (size_t)c * d.ldc] = d.B[r + (size_t)c * d.ldb];
}
void launch_copy_rows(const GemmDesc* d, int nb, int maxrows, int ncol, cudaStream_t s) {
    if (nb <= 0 || maxrows <= 0 || ncol <= 0) return;
    dim3 grid((maxrows * ncol + 255) / 256, 1, nb);
    k_copy_rows<<<grid, 256, 0, s>>>(d, ncol);
}

__global__ void k_convert_f32(const zd* __restrict__ src, zf* __restrict__ dst, size_t n) {
    const size_t i = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (i < n) dst[i] = tof(src[i]);
}
void launch_convert_f32(const zd* src, zf* dst, size_t n, cudaStream_t s) {
    if (n == 0) return;
    k_convert_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
}

__global__ void k_conj_transpose(const zd* __restrict__ A, zd* __restrict__ AT, int m, int n) {
    __shared__ zd t[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;  // bx over m (rows of A), by over n
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int r = bx + threadIdx.x, c = by + j;
        if (r < m && c < n) t[j][threadIdx.x] = A[r + (size_t)c * m];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int r = by + threadIdx.x, c = bx + j;  // AT[r, c] = conj(A[c, r])
        if (r < n && c < m) AT[r + (size_t)c * n] = zconj(t[threadIdx.x][j]);
    }
}
void launch_conj_transpose(const zd* A, zd* AT, int m, int n, cudaStream_t s) {
    if (m <= 0 || n <= 0) return;
    dim3 grid((m + 31) / 32, (n + 31) / 32), block(32, 8);
    k_conj_transpose<<<grid, block, 0, s>>>(A, AT, m, n);
}
