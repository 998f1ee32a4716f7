// The RT-TDDFT step in the auxiliary subspace (arXiv 2403.04351, Sec. 2):
//   HH(t_k)  = diag(eps) + (A_k/c).PP + |A_k|^2/(2c^2) I [+ dVV(t_k)]
//              (Eq. auxiliary_hamiltonian_with_parts, SS = I for the S-orthonormal basis)
//   theta'   = exp(-i HH dt) theta (Chebyshev or Jacobi eigen-decomposition) or the
//              Crank-Nicolson map (Eq. evolution_of_projection_coeff)
//   C        = CC theta'                                   (Eq. approximation_coefficients)
//   [HC|SC]  = H(A_k) C, S C from the submatrices           (Eq. v_MT, v_interstitial, App. A)
//   theta~   = CC^H S C                                    (projection coefficients)
//   J, dmu, E, C^H S C reduced per step                     (Eq. dipole)
#include <math.h>

#include "rtd.h"

#include <cstdlib>

__device__ __forceinline__ double dsq(double x) { return x * x; }

// ------------------------------------------------------------ step scalars
// A_k and s_k of the current step are copied into the device state so that
// every later kernel of the step reads them from one place.
__global__ void k_set_cur(StepArgs a) {
    DevState* st = a.st;
    const int cs = st->cstep;
    const double* av = a.a + 3 * (size_t)cs;
    st->cur_a[0] = av[0];
    st->cur_a[1] = av[1];
    st->cur_a[2] = av[2];
    st->cur_s = a.dvs ? a.dvs[cs] : (a.hartree ? 1.0 : 0.0);
    st->cur_aa = (av[0] * av[0] + av[1] * av[1] + av[2] * av[2]) * a.half_inv_c2;
}

// V~ + s dV~ (and its FP32 copy) for steps with a potential change
__global__ void k_vstep(StepArgs a) {
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= a.nvt) return;
    const double s = a.st->cur_s;
    const zd v = zadd(a.vtab[i], zscale(a.dvtab[i], s));
    a.vstep[i] = v;
    if (a.vstep32) a.vstep32[i] = tof(v);
    if (a.vsteps) {
        bool o1, o2;
        a.vsteps[i] = make_uint2(split16_bits(v.x, a.tc_fmt, a.tc_st, o1), split16_bits(v.y, a.tc_fmt, a.tc_st, o2));
        if (!(o1 && o2)) atomicOr(a.flag, 32);
    }
}

// ------------------------------------------------------------ HH(t_k)
// HH = diag(eps + |A|^2/(2c^2)) + sum_l (A_l/c) PP_l (+ dVV).  Without a
// potential change this kernel also stores the step's A and |A|^2/(2c^2)
// for the kernels that follow (with one, k_set_cur ran first).
__global__ void k_hsub(StepArgs a) {
    const KDev& K = a.kd[blockIdx.z];
    const int n = a.naux;
    DevState* st = a.st;
    const double* av = a.a + 3 * (size_t)st->cstep;
    const double ax = av[0], ay = av[1], az = av[2];
    const double aa = (ax * ax + ay * ay + az * az) * a.half_inv_c2;
    if (blockIdx.x == 0 && blockIdx.z == 0 && threadIdx.x == 0) {
        st->bar = 0u;
        if (!a.dv_on) {
            st->cur_a[0] = ax;
            st->cur_a[1] = ay;
            st->cur_a[2] = az;
            st->cur_s = 0.0;
            st->cur_aa = aa;
        }
    }
    const int idx = blockIdx.x * 256 + threadIdx.x;
    if (idx >= n * n) return;
    const int i = idx % n, j = idx / n;
    const size_t nn = (size_t)n * n;
    const double al[3] = {ax * a.inv_c, ay * a.inv_c, az * a.inv_c};
    zd v = zmk(0.0, 0.0);
#pragma unroll
    for (int l = 0; l < 3; ++l)
        if (al[l] != 0.0) v = zadd(v, zscale(K.psub[l * nn + idx], al[l]));
    if (i == j) v.x += K.eps[i] + aa;
    if (a.dv_on) v = zadd(v, K.dvsub[idx]);
    K.hsub[idx] = v;
}

// ------------------------------------------------------------ Chebyshev
// Term n of  sum_n c_n T_n(H~) theta,  H~ = (HH - lam_c)/lam_h:
//   y_1 = H~ y_0, y_n = 2 H~ y_{n-1} - y_{n-2}; acc += c_n y_n.
// One block per row i (threads over the columns of HH; HH is Hermitian so
// row i is read as the contiguous column i), so every SM shares the FP64 work.
template <int NT>
__global__ void __launch_bounds__(128) k_cheb(StepArgs a, int nt, int last) {
    __shared__ double red[4][2 * NT];
    const KDev& K = a.kd[blockIdx.z];
    const int n = a.naux, ns = a.ns;
    const int i = blockIdx.x;
    if (i >= n) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t vs = (size_t)n * ns;
    const zd* __restrict__ H = K.hsub + (size_t)i * n;
    const zd* yin = (nt == 1) ? K.theta : K.ring + ((nt - 1) % 3) * vs;
    const zd* yp2 = (nt >= 2) ? K.ring + ((nt - 2) % 3) * vs : nullptr;
    zd* yout = K.ring + (nt % 3) * vs;
    const double lc = K.lam[0], ilh = K.lam[2];
    const zd cn = K.coef[nt];
    for (int n0 = 0; n0 < ns; n0 += NT) {
        zd acc[NT];
#pragma unroll
        for (int c = 0; c < NT; ++c) acc[c] = zmk(0.0, 0.0);
        for (int j = tid; j < n; j += 128) {
            const zd h = H[j];
#pragma unroll
            for (int c = 0; c < NT; ++c)
                if (n0 + c < ns) zfmac(acc[c], h, yin[j + (size_t)(n0 + c) * n]);
        }
#pragma unroll
        for (int c = 0; c < NT; ++c) {
            const zd r = warp_zsum(acc[c]);
            if (lane == 0) {
                red[warp][2 * c] = r.x;
                red[warp][2 * c + 1] = r.y;
            }
        }
        __syncthreads();
        if (tid < NT && n0 + tid < ns) {
            const int c = tid;
            const zd v = zmk(red[0][2 * c] + red[1][2 * c] + red[2][2 * c] + red[3][2 * c],
                             red[0][2 * c + 1] + red[1][2 * c + 1] + red[2][2 * c + 1] + red[3][2 * c + 1]);
            const size_t e = i + (size_t)(n0 + c) * n;
            const zd yi = yin[e];
            const zd w = zscale(zsub(v, zscale(yi, lc)), ilh);
            zd y, ac;
            if (nt == 1) {
                y = w;
                K.ring[e] = yi;  // y_0
                ac = zadd(zmul(K.coef[0], yi), zmul(cn, y));
            } else {
                y = zsub(zscale(w, 2.0), yp2[e]);
                ac = zadd(K.acc[e], zmul(cn, y));
            }
            yout[e] = y;
            if (last) {
                // exp form: e^{-i dt lam_c}; Crank-Nicolson form: the centre is inside c_n
                const zd ph = (a.prop == 0) ? zmk(K.lam[3], K.lam[4]) : zmk(1.0, 0.0);
                K.theta[e] = zmul(ph, ac);
            } else {
                K.acc[e] = ac;
            }
        }
        __syncthreads();
    }
}

// Grid-wide barrier of a cooperative launch: a monotone arrival counter in
// device memory (zeroed by k_hsub before the launch); a block waits until
// the counter reaches `target`.  The wait is bounded: after about 0.3 s it
// raises flag bit 2 (reported as ERR_TIMEOUT) and returns false, so a launch
// can never hang.
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ bool grid_barrier(unsigned* count, unsigned target, int* flag) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        // release: the block's writes (ordered before by the bar.sync above)
        // become visible to every block that acquires the count
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(count), "r"(1u) : "memory");
        int ok = 1;
        unsigned long long it = 0;
        while (ld_acquire_gpu(count) < target) {
            if (++it > (1ull << 22)) {
                atomicOr(flag, 4);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The whole Chebyshev series in one cooperative launch.  A block of two
// warps owns rows (k, i) = blockIdx.x + r gridDim.x for all terms; its lanes
// stride a row's dot products and reduce them with WarpHalvingSum (the FP64
// pipe, not memory, bounds a term on GB300).  Only the newest vector y_{n-1}
// is exchanged through global memory (two slots, read through L2 with
// ld.global.cg); each block keeps y_{n-1}, y_{n-2} and the partial sum of
// its own rows in shared memory.  A grid barrier separates the terms (per-block
// epoch flags polled by every block measured slower on GB300: 107 against 80 us
// per series at N_aux = 200).
#define CHEB_THREADS 64
#define CHEB_JU 4  // row entries per thread held at once (n_aux <= 256 in one pass)
template <int NT>
__global__ void __launch_bounds__(CHEB_THREADS) k_cheb_coop(StepArgs a, int direct) {
    constexpr int V = 2 * NT;
    __shared__ double red[CHEB_THREADS / 32][V];
    extern __shared__ zd cst[];  // [rows of the block][3][ns]: y_{n-1}, y_{n-2}, partial sum
    const int n = a.naux, ns = a.ns;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t vs = (size_t)n * ns;
    const int nrow = a.nk * n;
    // direct: every block owns one row and n <= CHEB_JU * CHEB_THREADS, so the
    // block builds its row of HH(t_k) (Eq. auxiliary_hamiltonian_with_parts)
    // once, in registers, instead of reading a matrix formed by k_hsub
    zd hrow[CHEB_JU];
    if (direct && blockIdx.x < nrow) {
        const int k = blockIdx.x / n, i = blockIdx.x % n;
        const KDev& K = a.kd[k];
        DevState* st = a.st;
        const double* av = a.a + 3 * (size_t)st->cstep;
        const double ax = av[0], ay = av[1], az = av[2];
        const double aa = (ax * ax + ay * ay + az * az) * a.half_inv_c2;
        if (blockIdx.x == 0 && tid == 0 && !a.dv_on) {
            st->cur_a[0] = ax;
            st->cur_a[1] = ay;
            st->cur_a[2] = az;
            st->cur_s = 0.0;
            st->cur_aa = aa;
        }
        const size_t nn = (size_t)n * n;
        const double al[3] = {ax * a.inv_c, ay * a.inv_c, az * a.inv_c};
#pragma unroll
        for (int u = 0; u < CHEB_JU; ++u) {
            const int j = tid + u * CHEB_THREADS;
            zd v = zmk(0.0, 0.0);
            if (j < n) {
                const size_t e = (size_t)i * n + j;  // the storage element (row j, column i) of k_hsub
#pragma unroll
                for (int l = 0; l < 3; ++l)
                    if (al[l] != 0.0) v = zadd(v, zscale(K.psub[l * nn + e], al[l]));
                if (i == j) v.x += K.eps[i] + aa;
                if (a.dv_on) v = zadd(v, K.dvsub[e]);
            }
            hrow[u] = v;
        }
    }
    for (int nt = 1; nt < a.nterms; ++nt) {
        const int last = (nt == a.nterms - 1);
        int r = 0;
        for (int q = blockIdx.x; q < nrow; q += gridDim.x, ++r) {
            const int k = q / n, i = q % n;
            const KDev& K = a.kd[k];
            const zd* __restrict__ H = K.hsub + (size_t)i * n;
            const zd* yin = (nt == 1) ? K.theta : K.ring + ((nt - 1) & 1) * vs;
            zd* yout = K.ring + (nt & 1) * vs;
            zd* y1 = cst + (size_t)r * 3 * ns;
            zd* y2 = y1 + ns;
            zd* ac = y2 + ns;
            for (int n0 = 0; n0 < ns; n0 += NT) {
                // operands of the update first, so their latency overlaps the dot products
                const bool upd = tid < NT && n0 + tid < ns;
                zd yi = zmk(0.0, 0.0), cn = zmk(0.0, 0.0), c0 = zmk(0.0, 0.0);
                double lc = 0.0, ilh = 0.0;
                if (upd) {
                    yi = (nt == 1) ? K.theta[i + (size_t)(n0 + tid) * n] : y1[n0 + tid];
                    cn = K.coef[nt];
                    if (nt == 1) c0 = K.coef[0];
                    lc = K.lam[0];
                    ilh = K.lam[2];
                }
                zd acc[NT];
#pragma unroll
                for (int c = 0; c < NT; ++c) acc[c] = zmk(0.0, 0.0);
                for (int j0 = tid; j0 < n; j0 += CHEB_JU * CHEB_THREADS) {
                    zd hv[CHEB_JU], yv[CHEB_JU][NT];
#pragma unroll
                    for (int u = 0; u < CHEB_JU; ++u) {
                        const int j = j0 + u * CHEB_THREADS;
                        const bool ok = j < n;
                        hv[u] = direct ? hrow[u] : (ok ? H[j] : zmk(0.0, 0.0));
#pragma unroll
                        for (int c = 0; c < NT; ++c)
                            yv[u][c] = (ok && n0 + c < ns) ? __ldcg(yin + j + (size_t)(n0 + c) * n) : zmk(0.0, 0.0);
                    }
#pragma unroll
                    for (int u = 0; u < CHEB_JU; ++u)
#pragma unroll
                        for (int c = 0; c < NT; ++c) zfmac(acc[c], hv[u], yv[u][c]);
                }
                double v[V];
#pragma unroll
                for (int c = 0; c < NT; ++c) {
                    v[2 * c] = acc[c].x;
                    v[2 * c + 1] = acc[c].y;
                }
                warp_sum_store<double, V>(v, lane, red[warp]);
                __syncthreads();
                if (upd) {
                    const int c = n0 + tid;
                    zd sm = zmk(red[0][2 * tid], red[0][2 * tid + 1]);
#pragma unroll
                    for (int w = 1; w < CHEB_THREADS / 32; ++w) sm = zadd(sm, zmk(red[w][2 * tid], red[w][2 * tid + 1]));
                    const zd w = zscale(zsub(sm, zscale(yi, lc)), ilh);
                    zd y, s;
                    if (nt == 1) {
                        y = w;
                        s = zadd(zmul(c0, yi), zmul(cn, y));
                    } else {
                        y = zsub(zscale(w, 2.0), y2[c]);
                        s = zadd(ac[c], zmul(cn, y));
                    }
                    y2[c] = yi;
                    y1[c] = y;
                    if (last) {
                        const zd ph = (a.prop == 0) ? zmk(K.lam[3], K.lam[4]) : zmk(1.0, 0.0);
                        K.theta[i + (size_t)c * n] = zmul(ph, s);
                    } else {
                        yout[i + (size_t)c * n] = y;
                        ac[c] = s;
                    }
                }
                __syncthreads();
            }
        }
        if (!last && !grid_barrier(&a.st->bar, (unsigned)nt * gridDim.x, a.flag)) return;
    }
}

// The series for many states (4 < N_s <= 64): a block owns a tile of CT_ROWS
// rows of HH (kept in shared memory for the whole series) and all the
// columns; a thread accumulates one row x CT_PER columns over the full dot
// product (independent FMA chains, no cross-lane sums), with y_{n-1} staged
// through shared memory in chunks of CT_KC rows.  One tile per block, so the
// per-output recurrence state (y_{n-1}, y_{n-2}, partial sum) stays in
// registers across the terms.
#define CT_ROWS 8
#define CT_THREADS 128
#define CT_COLS 64
#define CT_PER (CT_COLS * CT_ROWS / CT_THREADS)
#define CT_KC 16
#define CT_YS (CT_COLS + 1)  // padded row of the staged chunk
static size_t cheb_tile_smem(int n) { return ((size_t)CT_ROWS * n + (size_t)CT_KC * CT_YS) * sizeof(zd); }

__global__ void __launch_bounds__(CT_THREADS) k_cheb_tile(StepArgs a) {
    extern __shared__ __align__(16) unsigned char ctsm[];
    const int n = a.naux, ns = a.ns;
    zd* Hs = (zd*)ctsm;                      // [CT_ROWS][n]
    zd* Ys = Hs + (size_t)CT_ROWS * n;       // [CT_KC][CT_YS]
    const int tpk = (n + CT_ROWS - 1) / CT_ROWS;
    const int k = blockIdx.x / tpk, i0 = (blockIdx.x - k * tpk) * CT_ROWS;
    const KDev& K = a.kd[k];
    const int tid = threadIdx.x;
    const int r = tid / (CT_COLS / CT_PER), cg = tid - r * (CT_COLS / CT_PER);
    const int i = i0 + r;
    const bool rok = i < n;
    const size_t vs = (size_t)n * ns;
    for (int e = tid; e < CT_ROWS * n; e += CT_THREADS) {
        const int rr = e / n, j = e - rr * n;
        Hs[e] = (i0 + rr < n) ? K.hsub[(size_t)(i0 + rr) * n + j] : zmk(0.0, 0.0);
    }
    zd y1[CT_PER], y2[CT_PER], ac[CT_PER];
#pragma unroll
    for (int u = 0; u < CT_PER; ++u) y1[u] = y2[u] = ac[u] = zmk(0.0, 0.0);
    const double lc = K.lam[0], ilh = K.lam[2];
    for (int nt = 1; nt < a.nterms; ++nt) {
        const int last = (nt == a.nterms - 1);
        const zd* yin = (nt == 1) ? K.theta : K.ring + ((nt - 1) & 1) * vs;
        zd* yout = K.ring + (nt & 1) * vs;
        zd acc[CT_PER];
#pragma unroll
        for (int u = 0; u < CT_PER; ++u) acc[u] = zmk(0.0, 0.0);
        for (int kc = 0; kc < n; kc += CT_KC) {
            __syncthreads();  // the previous chunk (or the H tile) is complete
            for (int e = tid; e < CT_KC * CT_COLS; e += CT_THREADS) {
                const int jj = e % CT_KC, c = e / CT_KC;
                Ys[jj * CT_YS + c] = (kc + jj < n && c < ns) ? __ldcg(yin + kc + jj + (size_t)c * n) : zmk(0.0, 0.0);
            }
            __syncthreads();
            const int jm = min(CT_KC, n - kc);
            const zd* hr = Hs + (size_t)r * n + kc;
            for (int jj = 0; jj < jm; ++jj) {
                const zd h = hr[jj];
#pragma unroll
                for (int u = 0; u < CT_PER; ++u) zfmac(acc[u], h, Ys[jj * CT_YS + cg + u * (CT_COLS / CT_PER)]);
            }
        }
        const zd cn = K.coef[nt];
        const zd c0 = K.coef[0];
        zd out[CT_PER];
#pragma unroll
        for (int u = 0; u < CT_PER; ++u) {
            const int c = cg + u * (CT_COLS / CT_PER);
            out[u] = zmk(0.0, 0.0);
            if (!rok || c >= ns) continue;
            const zd yi = (nt == 1) ? K.theta[i + (size_t)c * n] : y1[u];
            const zd w = zscale(zsub(acc[u], zscale(yi, lc)), ilh);
            zd y, sm;
            if (nt == 1) {
                y = w;
                sm = zadd(zmul(c0, yi), zmul(cn, y));
            } else {
                y = zsub(zscale(w, 2.0), y2[u]);
                sm = zadd(ac[u], zmul(cn, y));
            }
            y2[u] = yi;
            y1[u] = y;
            ac[u] = sm;
            out[u] = y;
        }
        if (last) {
            // theta is the input of the first term: with a two-term series wait for every block
            if (nt == 1 && !grid_barrier(&a.st->bar, (unsigned)nt * gridDim.x, a.flag)) return;
            const zd ph = (a.prop == 0) ? zmk(K.lam[3], K.lam[4]) : zmk(1.0, 0.0);
#pragma unroll
            for (int u = 0; u < CT_PER; ++u) {
                const int c = cg + u * (CT_COLS / CT_PER);
                if (rok && c < ns) K.theta[i + (size_t)c * n] = zmul(ph, ac[u]);
            }
        } else {
#pragma unroll
            for (int u = 0; u < CT_PER; ++u) {
                const int c = cg + u * (CT_COLS / CT_PER);
                if (rok && c < ns) yout[i + (size_t)c * n] = out[u];
            }
            if (!grid_barrier(&a.st->bar, (unsigned)nt * gridDim.x, a.flag)) return;
        }
    }
}

// Chebyshev coefficients of the call, per k-point.
//  exp:  e^{-i z x} = sum_n eps_n (-i)^n J_n(z) T_n(x), z = dt lam_h (Jacobi-Anger);
//        J_n(z) by Miller's backward recurrence normalised with J_0 + 2 sum J_2m = 1.
//  CN:   f(x) = (1 - i dt/2 (lc + lh x)) / (1 + i dt/2 (lc + lh x)) projected on
//        T_n by the discrete cosine sums at 256 Chebyshev points.
__global__ void k_coef(StepArgs a) {
    const KDev& K = a.kd[blockIdx.x];
    const int nt = a.nterms;
    const double lc = K.lam[0], lh = K.lam[1];
    if (a.prop == 0) {
        if (threadIdx.x != 0) return;
        const double z = a.dt * lh;
        zd* c = K.coef;
        if (z < 1e-300) {
            c[0] = zmk(1.0, 0.0);
            for (int q = 1; q < nt; ++q) c[q] = zmk(0.0, 0.0);
            return;
        }
        const int big = (nt > (int)z ? nt : (int)z);
        int M = big + 20 + (int)sqrt(40.0 * big);
        if (M & 1) ++M;
        double jp = 0.0, jc = 1.0, sum = 0.0;  // J_{M+1}, J_M (unnormalised)
        for (int q = 0; q < nt; ++q) c[q].x = 0.0;
        for (int m = M; m >= 1; --m) {
            const double jn = (2.0 * m / z) * jc - jp;
            jp = jc;
            jc = jn;
            const int idx = m - 1;
            if (idx < nt) c[idx].x = jc;
            if (idx >= 2 && (idx & 1) == 0) sum += 2.0 * jc;
            if (fabs(jc) > 1e200) {
                jc *= 1e-200;
                jp *= 1e-200;
                sum *= 1e-200;
                for (int q = idx; q < nt; ++q) c[q].x *= 1e-200;
            }
        }
        sum += jc;
        for (int q = 0; q < nt; ++q) {
            const double jq = c[q].x / sum;
            const double e = (q == 0) ? 1.0 : 2.0;
            zd v;
            switch (q & 3) {
                case 0: v = zmk(e * jq, 0.0); break;
                case 1: v = zmk(0.0, -e * jq); break;
                case 2: v = zmk(-e * jq, 0.0); break;
                default: v = zmk(0.0, e * jq); break;
            }
            c[q] = v;
        }
    } else {
        // one warp: c_q = (2 - delta_q0)/P sum_j f(x_j) cos(q th_j), th_j = pi (j + 1/2)/P
        const int P = 256;
        const int lane = threadIdx.x & 31;
        if (threadIdx.x >= 32) return;
        const double hd = 0.5 * a.dt;
        for (int q = 0; q < nt; ++q) {
            zd s = zmk(0.0, 0.0);
            for (int j = lane; j < P; j += 32) {
                const double th = M_PI * (j + 0.5) / P;
                const double lam = lc + lh * cos(th);
                const double u = hd * lam;
                // (1 - i u) / (1 + i u) = ((1 - u^2) - 2 i u) / (1 + u^2)
                const double den = 1.0 + u * u;
                const zd f = zmk((1.0 - u * u) / den, -2.0 * u / den);
                s = zadd(s, zscale(f, cos(q * th)));
            }
            s = warp_zsum(s);
            if (lane == 0) K.coef[q] = zscale(s, (q == 0 ? 1.0 : 2.0) / P);
        }
    }
}

// ------------------------------------------------------------ operator pass
// Local (muffin-tin) stage, one warp per local row i of atom alpha:
//   Z_H = h_eff X_loc,  Z_S = o X_loc,  h_eff = h + (A/c).p + |A|^2/(2c^2) o + s dh
// with X_loc = [A_alpha C_G ; C_lo(alpha)] (Eq. v_MT with the block map
// [A 0; 0 I]); the matching rows go to Z (back-projected next), the LO rows
// directly into [HC | SC].  Per row it also stores sum_n f_n Re x^* (p_l X)
// (the muffin-tin part of c^H P c) and, for LO rows, the rows' share of
// c^H H c and c^H S c.
template <typename TC, int NT>
__global__ void __launch_bounds__(32) k_local(StepArgs a) {
    using R = decltype(TC{}.x);
    constexpr bool F32 = sizeof(R) == 4;
    constexpr int VP = (10 * NT <= 32) ? 32 : 64;  // 5 complex sums per column, padded
    __shared__ R red[VP];
    const int k = blockIdx.z;
    const KDev& K = a.kd[k];
    const AtomTab& at = *a.at;
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x;
    if (row >= at.lrows) return;
    int al = 0;
    while (al + 1 < at.n && at.loff[al + 1] <= row) ++al;
    const int i = row - at.loff[al];
    const int m = at.m[al], na = at.na[al];
    const size_t mm = (size_t)m * m;
    const size_t boff = at.boff[al] + (size_t)i * m;
    const zd* __restrict__ dh = a.dh ? a.dh + boff : nullptr;
    const DevState* st = a.st;
    const double cx = st->cur_a[0] * a.inv_c, cy = st->cur_a[1] * a.inv_c, cz = st->cur_a[2] * a.inv_c;
    const double aa = st->cur_aa, sdv = st->cur_s;
    const int ns = a.ns, nb = K.nb, ma = at.ma, ng = K.ng;
    const int aoff = at.aoff[al], lo0 = ng + at.looff[al];
    double jc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int n0 = 0; n0 < ns; n0 += NT) {
        TC aH[NT], aS[NT], aP[3][NT];
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            aH[j] = aS[j] = Cx<TC>::zero();
            aP[0][j] = aP[1][j] = aP[2][j] = Cx<TC>::zero();
        }
        for (int jj = lane; jj < m; jj += 32) {
            TC hec, ojc, pxc, pyc, pzc;
            if constexpr (F32) {
                // the FP32 forms combine H(t) = h + A/c.p + |A|^2/2c^2 o in FP32
                const zf hj = a.h32[boff + jj], oj = a.o32[boff + jj];
                pxc = a.p32[3 * at.boff[al] + (size_t)i * m + jj];
                pyc = a.p32[3 * at.boff[al] + mm + (size_t)i * m + jj];
                pzc = a.p32[3 * at.boff[al] + 2 * mm + (size_t)i * m + jj];
                const float fx = (float)cx, fy = (float)cy, fz = (float)cz, fa = (float)aa;
                hec.x = hj.x + fx * pxc.x + fy * pyc.x + fz * pzc.x + fa * oj.x;
                hec.y = hj.y + fx * pxc.y + fy * pyc.y + fz * pzc.y + fa * oj.y;
                if (dh && sdv != 0.0) {
                    const zd d = dh[jj];
                    hec.x += (float)(sdv * d.x);
                    hec.y += (float)(sdv * d.y);
                }
                ojc = oj;
            } else {
                const zd* __restrict__ p = a.p + 3 * at.boff[al] + (size_t)i * m;
                const zd hj = a.h[boff + jj], oj = a.o[boff + jj];
                const zd px = p[jj], py = p[mm + jj], pz = p[2 * mm + jj];
                zd he = zadd(hj, zadd(zadd(zscale(px, cx), zscale(py, cy)), zadd(zscale(pz, cz), zscale(oj, aa))));
                if (dh && sdv != 0.0) he = zadd(he, zscale(dh[jj], sdv));
                hec = he;
                ojc = oj;
                pxc = px;
                pyc = py;
                pzc = pz;
            }
            const zd* xs = (jj < na) ? (K.Q + aoff + jj) : (K.C + lo0 + (jj - na));
            const size_t ld = (jj < na) ? (size_t)ma : (size_t)nb;
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                if (n0 + j >= ns) break;
                const TC x = Cx<TC>::from(xs[(size_t)(n0 + j) * ld]);
                Cx<TC>::fmac(aH[j], hec, x);
                Cx<TC>::fmac(aS[j], ojc, x);
                Cx<TC>::fmac(aP[0][j], pxc, x);
                Cx<TC>::fmac(aP[1][j], pyc, x);
                Cx<TC>::fmac(aP[2][j], pzc, x);
            }
        }
        R v[VP];
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            v[10 * j + 0] = aH[j].x;
            v[10 * j + 1] = aH[j].y;
            v[10 * j + 2] = aS[j].x;
            v[10 * j + 3] = aS[j].y;
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                v[10 * j + 4 + 2 * l] = aP[l][j].x;
                v[10 * j + 5 + 2 * l] = aP[l][j].y;
            }
        }
#pragma unroll
        for (int e = 10 * NT; e < VP; ++e) v[e] = (R)0;
        warp_sum_store<R, VP>(v, lane, red);
        __syncwarp();
        if (lane == 0) {
            for (int j = 0; j < NT; ++j) {
                const int c = n0 + j;
                if (c >= ns) break;
                const zd zh = zmk((double)red[10 * j], (double)red[10 * j + 1]);
                const zd zs = zmk((double)red[10 * j + 2], (double)red[10 * j + 3]);
                const zd q0 = zmk((double)red[10 * j + 4], (double)red[10 * j + 5]);
                const zd q1 = zmk((double)red[10 * j + 6], (double)red[10 * j + 7]);
                const zd q2 = zmk((double)red[10 * j + 8], (double)red[10 * j + 9]);
                zd xi;
                const double f = a.occ[c];
                if (i < na) {
                    K.Z[aoff + i + (size_t)c * ma] = zh;
                    K.Z[aoff + i + (size_t)(ns + c) * ma] = zs;
                    xi = K.Q[aoff + i + (size_t)c * ma];
                } else {
                    const int r = lo0 + (i - na);
                    K.Y[r + (size_t)c * nb] = zh;
                    K.Y[r + (size_t)(ns + c) * nb] = zs;
                    xi = K.C[r + (size_t)c * nb];
                    jc[3] += f * (xi.x * zh.x + xi.y * zh.y);
                    jc[4] += f * (xi.x * zs.x + xi.y * zs.y);
                }
                jc[0] += f * (xi.x * q0.x + xi.y * q0.y);
                jc[1] += f * (xi.x * q1.x + xi.y * q1.y);
                jc[2] += f * (xi.x * q2.x + xi.y * q2.y);
            }
        }
        __syncwarp();
    }
    if (lane == 0) {
        double* pj = a.part_jmt + ((size_t)k * at.lrows + row) * 5;
#pragma unroll
        for (int q = 0; q < 5; ++q) pj[q] = jc[q];
    }
}

// The muffin-tin products for many states (FP32 forms, N_s > 4): one block of
// four warps per (atom, chunk of its rows, k); X = [Q_a; C_lo,a] (m x N_s) is
// staged once in shared memory as FP32, lanes own columns (CPL per lane) and
// a warp walks one local row at a time, reading the row of h, o, p (FP32
// copies, broadcast) once for all columns.  Outputs as k_local.
#define LOCW_MIN_NS 16  // above this many states the columns-per-lane kernel wins
template <int CPL>
__global__ void __launch_bounds__(128) k_local_wide(StepArgs a, int rowchunks) {
    extern __shared__ zf xs[];  // [m][ns]
    const int k = blockIdx.z;
    const KDev& K = a.kd[k];
    const AtomTab& at = *a.at;
    const int al = blockIdx.x / rowchunks, chunk = blockIdx.x % rowchunks;
    if (al >= at.n) return;
    const int m = at.m[al], na = at.na[al];
    const int ns = a.ns, nb = K.nb, ma = at.ma, ng = K.ng;
    const int aoff = at.aoff[al], lo0 = ng + at.looff[al];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < m * ns; e += blockDim.x) {
        const int j = e / ns, c = e % ns;
        const zd x = (j < na) ? K.Q[aoff + j + (size_t)c * ma] : K.C[lo0 + (j - na) + (size_t)c * nb];
        xs[e] = tof(x);
    }
    __syncthreads();
    const DevState* st = a.st;
    const float fx = (float)(st->cur_a[0] * a.inv_c), fy = (float)(st->cur_a[1] * a.inv_c),
                fz = (float)(st->cur_a[2] * a.inv_c), fa = (float)st->cur_aa;
    const double sdv = st->cur_s;
    const size_t mm = (size_t)m * m;
    const int r0 = chunk * ((m + rowchunks - 1) / rowchunks);
    const int r1 = min(m, r0 + (m + rowchunks - 1) / rowchunks);
    for (int i = r0 + warp; i < r1; i += 4) {
        const size_t bo = at.boff[al] + (size_t)i * m;
        const zf* __restrict__ hr = a.h32 + bo;
        const zf* __restrict__ orow = a.o32 + bo;
        const zf* __restrict__ pr = a.p32 + 3 * at.boff[al] + (size_t)i * m;
        const zd* __restrict__ dh = a.dh ? a.dh + bo : nullptr;
        zf aH[CPL], aS[CPL], aP[3][CPL];
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            aH[q] = aS[q] = make_float2(0.f, 0.f);
            aP[0][q] = aP[1][q] = aP[2][q] = make_float2(0.f, 0.f);
        }
        for (int j = 0; j < m; ++j) {
            const zf hj = hr[j], oj = orow[j];
            const zf px = pr[j], py = pr[mm + j], pz = pr[2 * mm + j];
            zf he;
            he.x = hj.x + fx * px.x + fy * py.x + fz * pz.x + fa * oj.x;
            he.y = hj.y + fx * px.y + fy * py.y + fz * pz.y + fa * oj.y;
            if (dh && sdv != 0.0) {
                const zd d = dh[j];
                he.x += (float)(sdv * d.x);
                he.y += (float)(sdv * d.y);
            }
            const zf* xr = xs + (size_t)j * ns;
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
                const int c = lane + 32 * q;
                if (c < ns) {
                    const zf x = xr[c];
                    cfmac(aH[q], he, x);
                    cfmac(aS[q], oj, x);
                    cfmac(aP[0][q], px, x);
                    cfmac(aP[1][q], py, x);
                    cfmac(aP[2][q], pz, x);
                }
            }
        }
        // outputs and the row's occupation-weighted shares
        float jc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            const int c = lane + 32 * q;
            if (c >= ns) continue;
            const zd zh = tod(aH[q]), zs = tod(aS[q]);
            const zf xi = xs[(size_t)i * ns + c];
            const float f = (float)a.occ[c];
            if (i < na) {
                K.Z[aoff + i + (size_t)c * ma] = zh;
                K.Z[aoff + i + (size_t)(ns + c) * ma] = zs;
            } else {
                const int r = lo0 + (i - na);
                K.Y[r + (size_t)c * nb] = zh;
                K.Y[r + (size_t)(ns + c) * nb] = zs;
                jc[3] += f * (xi.x * aH[q].x + xi.y * aH[q].y);
                jc[4] += f * (xi.x * aS[q].x + xi.y * aS[q].y);
            }
#pragma unroll
            for (int l = 0; l < 3; ++l) jc[l] += f * (xi.x * aP[l][q].x + xi.y * aP[l][q].y);
        }
        float v[8] = {jc[0], jc[1], jc[2], jc[3], jc[4], 0.f, 0.f, 0.f};
        __shared__ float red[4][8];
        warp_sum_store<float, 8>(v, lane, red[warp]);
        __syncwarp();
        if (lane == 0) {
            double* pj = a.part_jmt + ((size_t)k * at.lrows + at.loff[al] + i) * 5;
#pragma unroll
            for (int q = 0; q < 5; ++q) pj[q] = (double)red[warp][q];
        }
        __syncwarp();
    }
}

// Muffin-tin blocks as GEMMs (FP32 forms, many states).  Per atom the stack
// G = [h_eff; o; p_x; p_y; p_z] (5m x m, column-major) with
// h_eff = h + (A/c).p + |A|^2/(2c^2) o (+ s dh) is formed once per step (it
// does not depend on k); the right-hand block [Q; C_lo] of every (k, atom) is
// gathered contiguous, W = G [Q; C_lo] is one batched tiled GEMM, and
// k_mt_epi distributes W:
// the h_eff and o rows go to Z (matching rows) or to the LO rows of
// [HC | SC], and the row's occupation-weighted shares of J (p rows) and of
// E and c^H S c (LO rows) go to part_jmt as in k_local.
__global__ void k_mt_form(StepArgs a) {
    const AtomTab& at = *a.at;
    const int al = blockIdx.y;
    if (al >= at.n) return;
    const int m = at.m[al];
    const size_t mm = (size_t)m * m, bo = at.boff[al];
    const DevState* st = a.st;
    const float fx = (float)(st->cur_a[0] * a.inv_c), fy = (float)(st->cur_a[1] * a.inv_c),
                fz = (float)(st->cur_a[2] * a.inv_c), fa = (float)st->cur_aa;
    const double sdv = st->cur_s;
    zf* G = a.mtg + 5 * bo;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < mm; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % m), j = (int)(e / m);  // element (i, j), column-major
        const zf hv = a.h32[bo + e], ov = a.o32[bo + e];
        const zf px = a.p32[3 * bo + e], py = a.p32[3 * bo + mm + e], pz = a.p32[3 * bo + 2 * mm + e];
        zf he;
        he.x = hv.x + fx * px.x + fy * py.x + fz * pz.x + fa * ov.x;
        he.y = hv.y + fx * px.y + fy * py.y + fz * pz.y + fa * ov.y;
        if (a.dh && sdv != 0.0) {
            const zd d = a.dh[bo + e];
            he.x += (float)(sdv * d.x);
            he.y += (float)(sdv * d.y);
        }
        zf* col = G + (size_t)j * 5 * m;
        col[i] = he;
        col[m + i] = ov;
        col[2 * m + i] = px;
        col[3 * m + i] = py;
        col[4 * m + i] = pz;
    }
}

// the right-hand block [Q_alpha; C_lo,alpha] of every (k, atom), contiguous
__global__ void k_mt_gather(StepArgs a) {
    const int k = blockIdx.z, al = blockIdx.y;
    const AtomTab& at = *a.at;
    if (al >= at.n) return;
    const KDev& K = a.kd[k];
    const int m = at.m[al], na = at.na[al], ns = a.ns;
    const int aoff = at.aoff[al], lo0 = K.ng + at.looff[al];
    zd* V = a.mtv + ((size_t)(a.kofs + k) * at.n + al) * a.mtv_stride;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * ns; e += gridDim.x * blockDim.x) {
        const int i = e % m, c = e / m;
        V[e] = (i < na) ? K.Q[aoff + i + (size_t)c * at.ma] : K.C[lo0 + (i - na) + (size_t)c * K.nb];
    }
}

__global__ void __launch_bounds__(128) k_mt_epi(StepArgs a) {
    const int k = blockIdx.z, al = blockIdx.y;
    const AtomTab& at = *a.at;
    if (al >= at.n) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int m = at.m[al], na = at.na[al];
    if (i >= m) return;
    const KDev& K = a.kd[k];
    const int ns = a.ns, nb = K.nb, ma = at.ma, ng = K.ng;
    const int aoff = at.aoff[al], lo0 = ng + at.looff[al];
    const size_t ent = (size_t)(a.kofs + k) * at.n + al;  // kofs: single-k operator calls
    const zd* W = a.mtw + ent * a.mtw_stride;
    const zd* V = a.mtv + ent * a.mtv_stride;
    const size_t ld = (size_t)5 * m;
    double jc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int c = 0; c < ns; ++c) {
        const zd* w = W + (size_t)c * ld;
        const zd zh = w[i], zs = w[m + i];
        const zd x = V[i + (size_t)c * m];
        const double f = a.occ[c];
        if (i < na) {
            K.Z[aoff + i + (size_t)c * ma] = zh;
            K.Z[aoff + i + (size_t)(ns + c) * ma] = zs;
        } else {
            const int r = lo0 + (i - na);
            K.Y[r + (size_t)c * nb] = zh;
            K.Y[r + (size_t)(ns + c) * nb] = zs;
            jc[3] += f * (x.x * zh.x + x.y * zh.y);
            jc[4] += f * (x.x * zs.x + x.y * zs.y);
        }
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const zd pv = w[(2 + l) * m + i];
            jc[l] += f * (x.x * pv.x + x.y * pv.y);
        }
    }
    double* pj = a.part_jmt + ((size_t)k * at.lrows + at.loff[al] + i) * 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) pj[q] = jc[q];
}

static int launch_mt_gemm(const StepArgs& a, const StepPlan& p, cudaStream_t s) {
    if (p.tcmt) {
        // split-BF16 form: the stacks formed in FP64 and the products on the tensor cores
        k_mt_gather<<<dim3((a.at_maxm * a.ns + 255) / 256, a.at_n, a.nk), 256, 0, s>>>(a);
        const int nl = launch_tc_mt(p.tcmt, a, s);
        k_mt_epi<<<dim3((a.at_maxm + 127) / 128, a.at_n, a.nk), 128, 0, s>>>(a);
        return nl + 2;
    }
    k_mt_form<<<dim3(64, a.at_n), 256, 0, s>>>(a);
    k_mt_gather<<<dim3((a.at_maxm * a.ns + 255) / 256, a.at_n, a.nk), 256, 0, s>>>(a);
    launch_gemm_nn(p.gd_mt1, a.nk * a.at_n, 5 * a.at_maxm, a.at_maxm, a.ns, 0, nullptr, 0, true, nullptr, s);
    k_mt_epi<<<dim3((a.at_maxm + 127) / 128, a.at_n, a.nk), 128, 0, s>>>(a);
    return 4;
}

// Plane-wave rows of H C and S C in independent partial sums, one block per
// (row tile of BT rows G, slot):
//  - slots 0 .. nseg-1: the interstitial sum of Eq. v_interstitial over one
//    segment of G',  T[G, n] = sum_{G' in segment} V~_{G-G'} C_G'.  G is listed
//    in lexicographic order, so the table offsets glin(G) - glin(G') of a
//    (row tile, column tile) pair form one contiguous window; the window and
//    the column tile of C are staged in shared memory and the inner loop
//    reads shared memory only;
//  - slots nseg .. nseg+naseg-1: the back-projection (A^H Z_H, A^H Z_S) over
//    one chunk of the matching rows, A^H read coalesced over the block's rows.
// Each slot writes [H part | S part] for columns n0 .. n0+NT-1 into part_t.
template <typename TA, typename TT, typename TC, int NT>
__global__ void __launch_bounds__(BT) k_toep_seg(StepArgs a, int n0, int slot0) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int k = blockIdx.z;
    const KDev& K = a.kd[k];
    const int ng = K.ng;
    const int g0 = blockIdx.x * BT;
    const int slot = blockIdx.y + slot0;
    const int tid = threadIdx.x;
    const int g = g0 + tid;
    const bool act = g < ng;
    const int ns = a.ns, nb = K.nb, ma = a.ma;
    const int nc = min(NT, ns - n0);
    TC aH[NT], aS[NT];
#pragma unroll
    for (int c = 0; c < NT; ++c) aH[c] = aS[c] = Cx<TC>::zero();
    if (slot < a.nseg) {
        const int c_lo = slot * a.segw;
        if (g0 >= ng || c_lo >= ng) return;
        const int c_hi = min(ng, c_lo + a.segw);
        TC* xs = (TC*)smem;                 // [BT][NT]
        int* ls = (int*)(xs + BT * NT);     // [BT]
        TT* ws = (TT*)(ls + BT);            // table window
        const int* __restrict__ glin = K.glin;
        const zd* __restrict__ X = K.C;
        const TT* __restrict__ tab;
        if constexpr (sizeof(TT) == sizeof(zf))
            tab = (const TT*)(a.dv_on ? (const void*)a.vstep32 : (const void*)a.vtab32);
        else
            tab = (const TT*)(a.dv_on ? (const void*)a.vstep : (const void*)a.vtab);
        const int Lr0 = glin[g0], Lr1 = glin[min(g0 + BT, ng) - 1];
        const int Lrow = act ? glin[g] : Lr0;
        for (int c0 = c_lo; c0 < c_hi; c0 += BT) {
            const int cw = min(BT, c_hi - c0);
            const int Lc0 = glin[c0], Lc1 = glin[c0 + cw - 1];
            const int wlo = Lr0 - Lc1 + a.vt_center;
            const int wn = Lr1 - Lc0 + a.vt_center - wlo + 1;
            __syncthreads();
            if (tid < cw) {
                ls[tid] = glin[c0 + tid];
#pragma unroll
                for (int c = 0; c < NT; ++c)
                    xs[tid * NT + c] = (c < nc) ? Cx<TC>::from(X[(c0 + tid) + (size_t)(n0 + c) * nb]) : Cx<TC>::zero();
            }
            for (int e = tid; e < wn; e += BT) ws[e] = tab[wlo + e];
            __syncthreads();
            if (act) {
                const int base = Lrow + a.vt_center - wlo;
                for (int i = 0; i < cw; ++i) {
                    const TC v = Cx<TC>::from(ws[base - ls[i]]);
#pragma unroll
                    for (int c = 0; c < NT; ++c) Cx<TC>::fma(aH[c], v, xs[i * NT + c]);
                }
            }
        }
    } else {
        const int r_lo = (slot - a.nseg) * a.msegw;
        if (g0 >= ng || r_lo >= ma) return;
        const int r_hi = min(ma, r_lo + a.msegw);
        TC* zs = (TC*)smem;  // [msegw][2 NT]
        const zd* __restrict__ Z = K.Z;
        const TA* __restrict__ AT;
        if constexpr (sizeof(TA) == sizeof(zf)) AT = (const TA*)K.at32;
        else AT = (const TA*)K.at;
        for (int r = r_lo + tid; r < r_hi; r += BT) {
            const int q = r - r_lo;
#pragma unroll
            for (int c = 0; c < NT; ++c) {
                zs[q * 2 * NT + c] = (c < nc) ? Cx<TC>::from(Z[r + (size_t)(n0 + c) * ma]) : Cx<TC>::zero();
                zs[q * 2 * NT + NT + c] = (c < nc) ? Cx<TC>::from(Z[r + (size_t)(ns + n0 + c) * ma]) : Cx<TC>::zero();
            }
        }
        __syncthreads();
        if (act) {
            const TA* ap = AT + g;
            for (int r = r_lo; r < r_hi; ++r) {
                const TC av = Cx<TC>::from(ap[(size_t)r * ng]);
                const TC* zr = zs + (r - r_lo) * 2 * NT;
#pragma unroll
                for (int c = 0; c < NT; ++c) {
                    Cx<TC>::fma(aH[c], av, zr[c]);
                    Cx<TC>::fma(aS[c], av, zr[NT + c]);
                }
            }
        }
    }
    if (act) {
        zd* pt = a.part_t + (((size_t)k * a.nslot + slot) * 2 * NT) * a.maxng + g;
#pragma unroll
        for (int c = 0; c < NT; ++c) {
            if (c >= nc) break;
            pt[(size_t)c * a.maxng] = Cx<TC>::todbl(aH[c]);
            pt[(size_t)(NT + c) * a.maxng] = Cx<TC>::todbl(aS[c]);
        }
    }
}

// Plane-wave rows of [HC | SC] (one thread per row G):
//   HC_G = |G+k+A/c|^2/2 C_G + (sum of the slots' H parts)
//   SC_G = C_G + (sum of the back-projection slots' S parts)
// summed in a fixed slot order.  The block adds its rows' f-weighted shares of
// Re c^H HC, Re c^H SC and sum (G+k)|c|^2 into its slot of part_full.
template <int NT>
// Columns n0 .. n1-1: at most NT when the slot partials are read; all
// columns in one launch when both parts arrive whole (K.th and K.tb).
__global__ void __launch_bounds__(BKB) k_back(StepArgs a, int n0, int n1) {
    __shared__ double rs[8];
    const int k = blockIdx.z;
    const KDev& K = a.kd[k];
    const int ng = K.ng;
    const int g0 = blockIdx.x * BKB;
    if (g0 >= ng) return;
    const int tid = threadIdx.x;
    const int g = g0 + tid;
    const bool act = g < ng;
    const int ns = a.ns, nb = K.nb;
    const zd* __restrict__ X = K.C;
    double red[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (act) {
        const int nsg = (ng + a.segw - 1) / a.segw;
        const int nas = (a.ma + a.msegw - 1) / a.msegw;
        const DevState* st = a.st;
        const double* q = K.gk + 3 * (size_t)g;
        const double dg = 0.5 * (dsq(q[0] + st->cur_a[0] * a.inv_c) + dsq(q[1] + st->cur_a[1] * a.inv_c) +
                                 dsq(q[2] + st->cur_a[2] * a.inv_c));
        for (int cc = n0; cc < n1; ++cc) {
            const int c = cc - n0;  // column within the slot partials
            zd th = zmk(0.0, 0.0), ts = zmk(0.0, 0.0);
            // slot partials, loads issued four slots at a time (in slot order)
            const zd* pt = a.part_t + (((size_t)k * a.nslot) * 2 * NT + (c < NT ? c : 0)) * a.maxng + g;
            const size_t sst = (size_t)2 * NT * a.maxng;
            auto sum4 = [&](int s0, int s1, size_t off) {
                zd t = zmk(0.0, 0.0);
                for (int sg = s0; sg < s1; sg += 4) {
                    zd v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        v[u] = (sg + u < s1) ? pt[(size_t)(sg + u) * sst + off] : zmk(0.0, 0.0);
#pragma unroll
                    for (int u = 0; u < 4; ++u) t = zadd(t, v[u]);
                }
                return t;
            };
            if (a.ith) th = K.th[g + (size_t)(n0 + c) * ng];
            else th = sum4(0, nsg, 0);
            if (a.tcback) {
                th = zadd(th, K.tb[g + (size_t)(n0 + c) * ng]);
                ts = K.tb[g + (size_t)(ns + n0 + c) * ng];
            } else {
                th = zadd(th, sum4(a.nseg, a.nseg + nas, 0));
                ts = sum4(a.nseg, a.nseg + nas, (size_t)NT * a.maxng);
            }
            const zd x = X[g + (size_t)(n0 + c) * nb];
            const zd hv = zadd(th, zscale(x, dg));
            const zd sv = zadd(ts, x);
            K.Y[g + (size_t)(n0 + c) * nb] = hv;
            K.Y[g + (size_t)(ns + n0 + c) * nb] = sv;
            const double f = a.occ[n0 + c];
            const double w = f * (x.x * x.x + x.y * x.y);
            red[0] += f * (x.x * hv.x + x.y * hv.y);
            red[1] += f * (x.x * sv.x + x.y * sv.y);
            red[2] += q[0] * w;
            red[3] += q[1] * w;
            red[4] += q[2] * w;
        }
    }
    // one warp: halving sum of the five shares
    const int lane = tid & 31;
    double v[8] = {red[0], red[1], red[2], red[3], red[4], 0.0, 0.0, 0.0};
    warp_sum_store<double, 8>(v, lane, rs);
    __syncwarp();
    if (tid < 5) {
        double* pf = a.part_full + ((size_t)k * a.max_nback + blockIdx.x) * 5 + tid;
        *pf = (n0 == 0) ? rs[tid] : *pf + rs[tid];
    }
}

// Sum over the block; every thread receives the total (fixed order).
__device__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    for (int w = 0; w < nw; ++w) r += sh[w];
    return r;
}
__device__ double block_max(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    for (int w = 0; w < nw; ++w) r = fmax(r, sh[w]);
    return r;
}

// Per subspace row i and component l (one warp each): finish
// theta~ = CC^H S C from the split-K partials (l == 0: its deviation from
// theta and, for N_s <= 4, the row's share of theta^H theta~), and the
// row's share of J_sub,l = sum_n f_n Re theta_in^* ((PP_l + A_l/c) theta)_in.
__device__ void post_body(const StepArgs& a, int do_theta, int do_j);
// (the step's finalize stays a launch of its own: run by the last post block
// it measured slower, 30 against 25 us at h2_6000, with fewer threads)
__global__ void __launch_bounds__(128) k_post(StepArgs a, int do_theta, int do_j) { post_body(a, do_theta, do_j); }
__device__ void post_body(const StepArgs& a, int do_theta, int do_j) {
    // halving warp sums over up to 4 columns at a time (each warp-wide FP64 add
    // is costly on GB300); per-warp scratch for the sums
    __shared__ double ws[4][8];
    const int k = blockIdx.z;
    const KDev& K = a.kd[k];
    const int n = a.naux, ns = a.ns;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w = blockIdx.x * 4 + warp;
    if (w >= 3 * n) return;
    const int i = w / 3, l = w % 3;
    double* prow = a.part_post + ((size_t)k * n + i) * POST_STRIDE;
    if (do_theta && l == 0) {
        const GemmDesc d = a.gd_proj[k];
        const int nsp = (d.K + a.kc_proj - 1) / a.kc_proj;
        double res = 0.0;
        zd mine = zmk(0.0, 0.0);
        for (int c0 = 0; c0 < ns; c0 += 4) {
            double v[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                zd t = zmk(0.0, 0.0);
                if (c0 + q < ns)
                    for (int sp = lane; sp < nsp; sp += 32)
                        t = zadd(t, a.part_proj[d.part_off + ((size_t)sp * ns + c0 + q) * n + i]);
                v[2 * q] = t.x;
                v[2 * q + 1] = t.y;
            }
            warp_sum_store<double, 8>(v, lane, ws[warp]);
            __syncwarp();
            for (int q = 0; q < 4 && c0 + q < ns; ++q) {
                const int c = c0 + q;
                const zd t = zmk(ws[warp][2 * q], ws[warp][2 * q + 1]);
                if (lane == 0) K.theta_t[i + (size_t)c * n] = t;
                const zd dd = zsub(t, K.theta[i + (size_t)c * n]);
                res = fmax(res, dd.x * dd.x + dd.y * dd.y);
                if (lane == c) mine = t;
            }
            __syncwarp();
        }
        res = sqrt(res);
        if (ns <= 4) {
            // row i's share of theta^H theta~ (= C^H S C for C = CC theta)
            const int pq = lane, pp = pq % ns, qq = pq / ns;
            const double tx = __shfl_sync(0xffffffffu, mine.x, qq < 32 ? qq : 0);
            const double ty = __shfl_sync(0xffffffffu, mine.y, qq < 32 ? qq : 0);
            if (pq < ns * ns) {
                const zd tp = K.theta[i + (size_t)pp * n];
                prow[4 + 2 * pq] = tp.x * tx + tp.y * ty;
                prow[4 + 2 * pq + 1] = tp.x * ty - tp.y * tx;
            }
        }
        if (lane == 0) prow[0] = res;
    }
    if (do_j) {
        const zd* __restrict__ P = K.psub + (size_t)l * n * n + (size_t)i * n;
        const double al = a.st->cur_a[l] * a.inv_c;
        double jl = 0.0;
        for (int c0 = 0; c0 < ns; c0 += 4) {
            double v[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                zd t = zmk(0.0, 0.0);
                if (c0 + q < ns) {
                    const zd* th = K.theta + (size_t)(c0 + q) * n;
                    for (int j = lane; j < n; j += 32) zfmac(t, P[j], th[j]);
                }
                v[2 * q] = t.x;
                v[2 * q + 1] = t.y;
            }
            warp_sum_store<double, 8>(v, lane, ws[warp]);
            __syncwarp();
            if (lane == 0) {
                for (int q = 0; q < 4 && c0 + q < ns; ++q) {
                    const int c = c0 + q;
                    const zd ti = K.theta[i + (size_t)c * n];
                    jl += a.occ[c] * (ti.x * (ws[warp][2 * q] + al * ti.x) + ti.y * (ws[warp][2 * q + 1] + al * ti.y));
                }
            }
            __syncwarp();
        }
        if (lane == 0) prow[1 + l] = jl;
    }
}

// The subspace current for many states through the occupation-weighted
// density matrix rho = theta F theta^H (F = diag(f)):
//   J_l = -(1/Omega) sum_k w_k [ Re tr(PP_l rho) + (A_l/c) tr(rho) ],
// the same quantity as sum_n f_n Re theta_n^H (PP_l + A_l/c) theta_n, at
// N_aux^2 (N_s / 2 + 3) complex products instead of 3 N_aux^2 N_s.  One block
// per pair of 32-row tiles (I <= J) of rho; rho is Hermitian and so is PP_l,
// so an off-diagonal pair counts twice (its mirror gives the conjugate).
// The block's three shares go to the J slots of row `pair` of part_post (the
// consumers sum those slots over rows); rows past the last pair get zeros.
#define JRHO_T 32
#define JRHO_CH 32
__global__ void __launch_bounds__(256) k_jrho(StepArgs a) {
    __shared__ zd sI[JRHO_CH][JRHO_T], sJ[JRHO_CH][JRHO_T];
    __shared__ double red[8][4];
    const int k = blockIdx.z;
    const KDev& K = a.kd[k];
    const int n = a.naux, ns = a.ns;
    const int nt = (n + JRHO_T - 1) / JRHO_T;
    const int npairs = nt * (nt + 1) / 2;
    const int pair = blockIdx.x;
    // pair -> (I, J), I <= J, row-major over the upper triangle
    int I = 0, rem = pair;
    while (rem >= nt - I) {
        rem -= nt - I;
        ++I;
    }
    const int J = I + rem;
    const int tid = threadIdx.x, i = tid & 31, jq = tid >> 5;
    const int gi = I * JRHO_T + i;
    zd acc[4] = {zmk(0.0, 0.0), zmk(0.0, 0.0), zmk(0.0, 0.0), zmk(0.0, 0.0)};
    for (int c0 = 0; c0 < ns; c0 += JRHO_CH) {
        __syncthreads();
        for (int e = tid; e < JRHO_CH * JRHO_T; e += 256) {
            const int cc = e >> 5, r = e & 31, c = c0 + cc;
            const int ri = I * JRHO_T + r, rj = J * JRHO_T + r;
            zd vi = zmk(0.0, 0.0), vj = zmk(0.0, 0.0);
            if (c < ns) {
                if (ri < n) vi = K.theta[ri + (size_t)c * n];
                if (rj < n) vj = zscale(K.theta[rj + (size_t)c * n], a.occ[c]);
            }
            sI[cc][r] = vi;
            sJ[cc][r] = vj;
        }
        __syncthreads();
        const int cn = min(JRHO_CH, ns - c0);
        for (int cc = 0; cc < cn; ++cc) {
            const zd ti = sI[cc][i];
#pragma unroll
            for (int q = 0; q < 4; ++q) zfmac(acc[q], ti, sJ[cc][jq + 8 * q]);  // rho[gj, gi] += f theta_gj conj(theta_gi)
        }
    }
    // shares of Re tr(PP_l rho) and of (A_l/c) tr(rho)
    double sh[3] = {0.0, 0.0, 0.0};
    const double wgt = (I == J) ? 1.0 : 2.0;
    if (gi < n) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gj = J * JRHO_T + jq + 8 * q;
            if (gj >= n) continue;
            for (int l = 0; l < 3; ++l) {
                const zd pp = K.psub[(size_t)l * n * n + gi + (size_t)gj * n];  // PP_l[gi, gj]
                double v = wgt * (pp.x * acc[q].x - pp.y * acc[q].y);
                if (gi == gj) v += a.st->cur_a[l] * a.inv_c * acc[q].x;
                sh[l] += v;
            }
        }
    }
    const int lane = tid & 31, warp = tid >> 5;
    for (int l = 0; l < 3; ++l) {
        const double v = warp_sum(sh[l]);
        if (lane == 0) red[warp][l] = v;
    }
    __syncthreads();
    if (tid < 3) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w][tid];
        a.part_post[((size_t)k * n + pair) * POST_STRIDE + 1 + tid] = t;
        for (int r = pair + npairs; r < n; r += npairs) a.part_post[((size_t)k * n + r) * POST_STRIDE + 1 + tid] = 0.0;
    }
}

// The post-projection launch(es): theta~ and its residual per row (do_theta),
// and the subspace current (do_j), by rows for few states and through the
// density matrix for many.
void launch_post(const StepArgs& a, int do_theta, int do_j, cudaStream_t s) {
    const bool rho = do_j && a.ns > JRHO_MIN_NS;
    if (do_theta || !rho) {
        dim3 g((3 * a.naux + 3) / 4, 1, a.nk);
        k_post<<<g, 128, 0, s>>>(a, do_theta, rho ? 0 : do_j);
    }
    if (rho) {
        const int nt = (a.naux + JRHO_T - 1) / JRHO_T;
        k_jrho<<<dim3(nt * (nt + 1) / 2, 1, a.nk), 256, 0, s>>>(a);
    }
}

// theta <- theta~ (3 I - theta~^H theta~) / 2: one Newton-Schulz step of the
// polar (Lowdin) factor, exact to O(|theta~^H theta~ - I|^2)
__global__ void k_reproj(StepArgs a) {
    const KDev& K = a.kd[blockIdx.z];
    const int ns = a.ns, n = a.naux;
    const int e = blockIdx.x * 256 + threadIdx.x;
    if (e >= n * ns) return;
    const int i = e % n, c = e / n;
    const zd* g2 = K.gram + (size_t)ns * ns;
    zd v = zmk(0.0, 0.0);
    for (int q = 0; q < ns; ++q) {
        zd w = zscale(g2[q + (size_t)c * ns], -0.5);
        if (q == c) w.x += 1.5;
        zfma(v, K.theta_t[i + (size_t)q * n], w);
    }
    K.theta[e] = v;
}

// Sum the step's partials over k-points (weights w_k) in a fixed order,
// update the dipole by the trapezoid rule (Eq. dipole) and append the
// record.  One block.
// First phase of the step's reductions: per (row chunk, k-point) block, the
// k-weighted sums of the per-row partials of the step (J_sub, E, c^H S c,
// sum (G+k)|c|^2, J_mt, the occupied ground-state share) and the maxima of
// the residual and of |C^H S C - I|, into part_fin[k][chunk].  The single
// block of k_finalize then sums these in (k, chunk) order.
// 0-2 J_sub, 3 E, 4 c^H S c, 5-7 sum (G+k)|c|^2, 8-10 J_mt, 11 occupied share, 12 max residual, 13 max dev
__global__ void __launch_bounds__(256) k_fin_part(StepArgs a, int set_gs) {
    __shared__ double sh[8][16];
    __shared__ unsigned long long shm[8][2];
    const int k = blockIdx.y, ch = blockIdx.x;
    const KDev& K = a.kd[k];
    const double w = a.wk[k];
    const int ns = a.ns, n = a.naux, lrows = a.lrows;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int nback = set_gs ? 0 : (K.ng + BKB - 1) / BKB;
    const int lr = set_gs ? 0 : lrows;
    const int cnt = max(n, max(nback, lr));
    double v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = 0.0;
    double mres = 0.0, mdev = 0.0;
    for (int i = ch * blockDim.x + tid; i < cnt; i += FIN_CH * blockDim.x) {
        double pp[4] = {0.0, 0.0, 0.0, 0.0}, pf[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, pj[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        if (i < n) {
            const double* p = a.part_post + ((size_t)k * n + i) * POST_STRIDE;
#pragma unroll
            for (int q = 0; q < 4; ++q) pp[q] = __ldcg(p + q);
        }
        if (i < nback) {
            const double* p = a.part_full + ((size_t)k * a.max_nback + i) * 5;
#pragma unroll
            for (int q = 0; q < 5; ++q) pf[q] = p[q];
        }
        if (i < lr) {
            const double* p = a.part_jmt + ((size_t)k * lrows + i) * 5;
#pragma unroll
            for (int q = 0; q < 5; ++q) pj[q] = p[q];
        }
        mres = fmax(mres, pp[0]);
        v[0] += w * pp[1];
        v[1] += w * pp[2];
        v[2] += w * pp[3];
#pragma unroll
        for (int q = 0; q < 5; ++q) v[3 + q] += w * pf[q];
        v[8] += w * pj[0];
        v[9] += w * pj[1];
        v[10] += w * pj[2];
        v[3] += w * pj[3];
        v[4] += w * pj[4];
    }
    if (!set_gs) {
        for (int e = ch * blockDim.x + tid; e < ns * ns; e += FIN_CH * blockDim.x) {
            const int i = e % ns, j = e / ns;
            const zd t = K.theta[i + (size_t)j * n];
            v[11] += w * a.occ[j] * (t.x * t.x + t.y * t.y);
        }
        if (ns <= 4) {
            // the rows' shares of theta^H theta~ in a fixed order (one warp per entry)
            __shared__ double gs[8][2];
            for (int e = ch * nw + warp; e < ns * ns; e += FIN_CH * nw) {
                double g[2] = {0.0, 0.0};
                for (int i = lane; i < n; i += 32) {
                    const double* p = a.part_post + ((size_t)k * n + i) * POST_STRIDE + 4 + 2 * e;
                    g[0] += __ldcg(p);
                    g[1] += __ldcg(p + 1);
                }
                warp_sum_store<double, 2>(g, lane, gs[warp]);
                __syncwarp();
                double gx = gs[warp][0];
                const double gy = gs[warp][1];
                if (e % ns == e / ns) gx -= 1.0;
                mdev = fmax(mdev, hypot(gx, gy));
                __syncwarp();
            }
        } else {
            for (int j = ch * blockDim.x + tid; j < ns; j += FIN_CH * blockDim.x)
                mdev = fmax(mdev, a.gdev[(size_t)k * ns + j]);
        }
    }
    warp_sum_store<double, 16>(v, lane, sh[warp]);
    unsigned long long br = (unsigned long long)__double_as_longlong(mres);
    unsigned long long bd = (unsigned long long)__double_as_longlong(mdev);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long xr = __shfl_xor_sync(0xffffffffu, br, o);
        const unsigned long long xd = __shfl_xor_sync(0xffffffffu, bd, o);
        br = xr > br ? xr : br;
        bd = xd > bd ? xd : bd;
    }
    if (lane == 0) {
        shm[warp][0] = br;
        shm[warp][1] = bd;
    }
    __syncthreads();
    double* out = a.part_fin + ((size_t)k * FIN_CH + ch) * FIN_STRIDE;
    if (tid < 12) {
        double t = sh[0][tid];
        for (int ww = 1; ww < nw; ++ww) t += sh[ww][tid];
        out[tid] = t;
    } else if (tid < 14) {
        unsigned long long m = shm[0][tid - 12];
        for (int ww = 1; ww < nw; ++ww) m = shm[ww][tid - 12] > m ? shm[ww][tid - 12] : m;
        out[tid] = __longlong_as_double((long long)m);
    }
}

// |C^H S C - I| for many states: column j of the gram theta^H theta~ per block
// (one warp per row i, lanes over the subspace rows), its largest deviation
// from the identity into gdev[k][j] (FP64).
__global__ void __launch_bounds__(256) k_gram_dev(StepArgs a) {
    __shared__ double wm[8];
    const int k = blockIdx.y, j = blockIdx.x;
    const KDev& K = a.kd[k];
    const int n = a.naux, ns = a.ns;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const zd* tt = K.theta_t + (size_t)j * n;
    double dev = 0.0;
    for (int i = warp; i < ns; i += 8) {
        const zd* th = K.theta + (size_t)i * n;
        zd g = zmk(0.0, 0.0);
        for (int r = lane; r < n; r += 32) zfmac(g, th[r], tt[r]);
        g = warp_zsum(g);
        if (i == j) g.x -= 1.0;
        dev = fmax(dev, hypot(g.x, g.y));
    }
    if (lane == 0) wm[warp] = dev;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = wm[0];
        for (int w = 1; w < 8; ++w) m = fmax(m, wm[w]);
        a.gdev[(size_t)k * ns + j] = m;
    }
}

__device__ void finalize_body(const StepArgs& a, int set_gs) {
    // the k-weights enter the per-row shares, so one block reduction covers all
    // k-points; sums by halving warp sums (each warp-wide FP64 add is costly on
    // GB300), maxima of non-negative values as integer maxima of their bits.
    // The kernel is latency-bound: every row's loads are issued before its adds,
    // and the scalars of the serial tail are fetched by the last warp meanwhile.
    __shared__ double sh[8][16];
    __shared__ unsigned long long shm[8][2];
    __shared__ double pre[16];  // 0 t, 1-3 A, 4-6 J(t0), 7-9 J_ind prev, 10-12 dmu, 13 dt_cr, 14 N_e
    __shared__ int pre_rec;
    DevState* st = a.st;
    const int ns = a.ns, n = a.naux, lrows = a.lrows;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    if (warp == nw - 1) {
        if (lane == 0) pre[0] = st->t;
        if (lane >= 1 && lane <= 3) pre[lane] = st->cur_a[lane - 1];
        if (lane >= 4 && lane <= 6) pre[lane] = st->j_gs[lane - 4];
        if (lane >= 7 && lane <= 9) pre[lane] = st->jind_prev[lane - 7];
        if (lane >= 10 && lane <= 12) pre[lane] = st->dmu[lane - 10];
        if (lane == 13) pre_rec = st->rec_count;
        if (!set_gs) {
            // dt_cr and N_e over the k-points, one lane per k
            double dtc = 1e300, ne = 0.0;
            for (int k = lane; k < a.nk; k += 32) {
                const KDev& K = a.kd[k];
                const double dk = (a.prop == 1) ? 0.2 / (K.eval[n - 1] - K.eval[0]) : 0.2 / (2.0 * K.lam[1]);
                dtc = fmin(dtc, dk);
                double f = 0.0;
                for (int j = 0; j < ns; ++j) f += a.occ[j];
                ne += a.wk[k] * f;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                dtc = fmin(dtc, __shfl_xor_sync(0xffffffffu, dtc, o));
                ne += __shfl_xor_sync(0xffffffffu, ne, o);
            }
            if (lane == 0) {
                pre[13] = dtc;
                pre[14] = ne;
            }
        }
    }
    // the per-(k, chunk) partials of k_fin_part, summed in (k, chunk) order
    double v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = 0.0;
    double mres = 0.0, mdev = 0.0;
    for (int e = tid; e < a.nk * FIN_CH; e += blockDim.x) {
        const double* p = a.part_fin + (size_t)e * FIN_STRIDE;
        double t[14];
#pragma unroll
        for (int q = 0; q < 14; ++q) t[q] = __ldcg(p + q);
#pragma unroll
        for (int q = 0; q < 12; ++q) v[q] += t[q];
        mres = fmax(mres, t[12]);
        mdev = fmax(mdev, t[13]);
    }
    warp_sum_store<double, 16>(v, lane, sh[warp]);
    unsigned long long br = (unsigned long long)__double_as_longlong(mres);
    unsigned long long bd = (unsigned long long)__double_as_longlong(mdev);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long xr = __shfl_xor_sync(0xffffffffu, br, o);
        const unsigned long long xd = __shfl_xor_sync(0xffffffffu, bd, o);
        br = xr > br ? xr : br;
        bd = xd > bd ? xd : bd;
    }
    if (lane == 0) {
        shm[warp][0] = br;
        shm[warp][1] = bd;
    }
    __syncthreads();
    if (tid < 12) {
        double t = sh[0][tid];
        for (int w = 1; w < nw; ++w) t += sh[w][tid];
        sh[0][tid] = t;
    } else if (tid < 14) {
        unsigned long long m = shm[0][tid - 12];
        for (int w = 1; w < nw; ++w) m = shm[w][tid - 12] > m ? shm[w][tid - 12] : m;
        shm[0][tid - 12] = m;
    }
    __syncthreads();
    if (tid != 0) return;
    const double io = -1.0 / a.omega;
    double J[3], JF[3];
    for (int l = 0; l < 3; ++l) {
        J[l] = io * sh[0][l];
        JF[l] = io * (sh[0][5 + l] + sh[0][8 + l] + pre[1 + l] * a.inv_c * sh[0][4]);
    }
    if (set_gs) {
        for (int l = 0; l < 3; ++l) st->j_gs[l] = J[l];
        return;
    }
    const double E = sh[0][3];
    const double res = __longlong_as_double((long long)shm[0][0]);
    const double ndev = __longlong_as_double((long long)shm[0][1]);
    const double t = pre[0] + a.dt;
    double* r = a.rec + (size_t)pre_rec * RTD_REC_STRIDE;
    r[REC_T] = t;
    for (int l = 0; l < 3; ++l) {
        const double jind = J[l] - pre[4 + l];
        const double dmu = pre[10 + l] + a.omega * a.dt * 0.5 * (pre[7 + l] + jind);
        st->dmu[l] = dmu;
        st->jind_prev[l] = jind;
        r[REC_J + l] = J[l];
        r[REC_JF + l] = JF[l];
        r[REC_DMU + l] = dmu;
    }
    r[REC_E] = E;
    // number of excited electrons: N_e minus the occupied ground-state share
    r[REC_NEXC] = pre[14] - sh[0][11];
    r[REC_NDEV] = ndev;
    r[REC_RES] = res;
    r[REC_DTCR] = pre[13];
    st->t = t;
    st->rec_count = pre_rec + 1;
    st->gstep += 1;
    st->cstep += 1;
    st->bar = 0u;  // the next step's cooperative series counts from zero
}

__global__ void __launch_bounds__(256) k_finalize(StepArgs a, int set_gs) { finalize_body(a, set_gs); }

void launch_finalize(const StepArgs& a, int set_gs, cudaStream_t s) {
    k_fin_part<<<dim3(FIN_CH, a.nk), 256, 0, s>>>(a, set_gs);
    k_finalize<<<1, 256, 0, s>>>(a, set_gs);
}


// ------------------------------------------------------------ Jacobi eigensolver
// Cyclic two-sided Jacobi for a complex Hermitian matrix (one block per
// matrix, matrix in global memory), with the round-robin ordering of the
// pairs so that each round applies n/2 independent rotations.  For the pair
// (p, q) with a_pq = r e^{i phi}: tau = (a_qq - a_pp)/(2r),
// t = sign(tau)/(|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c, and
// G = [[c, s], [-s e^{-i phi}, c e^{-i phi}]] on (p, q); A <- G^H A G,
// V <- V G.  Sweeps stop when the off-diagonal Frobenius norm is below
// 1e-15 of the total, or after max_sweeps (then *flag = 1).  Eigenvalues are
// returned ascending with the matching columns of V.
__global__ void __launch_bounds__(1024) k_jacobi(zd* const* mats, double* const* vals, zd* const* vecs,
                                                 int n, int max_sweeps, int* flag) {
    zd* A = mats[blockIdx.x];
    zd* V = vecs[blockIdx.x];
    double* w = vals[blockIdx.x];
    const int tid = threadIdx.x, nt = blockDim.x;
    const size_t nn = (size_t)n * n;
    __shared__ int sp[512], sq[512];
    __shared__ double sc[512], sv[512];
    __shared__ zd sph[512];
    __shared__ double sh[32];
    for (size_t e = tid; e < nn; e += nt) {
        const int i = (int)(e % n), j = (int)(e / n);
        V[e] = zmk(i == j ? 1.0 : 0.0, 0.0);
        if (i == j) A[e].y = 0.0;
    }
    __syncthreads();
    const int ne = n + (n & 1), np = ne / 2;
    int sweep = 0;
    bool conv = (n <= 1);
    for (; sweep < max_sweeps && !conv; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (size_t e = tid; e < nn; e += nt) {
            const zd v = A[e];
            const double m2 = v.x * v.x + v.y * v.y;
            tot += m2;
            if ((int)(e % n) != (int)(e / n)) off += m2;
        }
        off = block_sum(off, sh);
        tot = block_sum(tot, sh);
        if (off <= 1e-30 * tot || tot == 0.0) {
            conv = true;
            break;
        }
        for (int r = 0; r < ne - 1; ++r) {
            for (int t = tid; t < np; t += nt) {
                int p, q;
                if (t == 0) {
                    p = ne - 1;
                    q = r;
                } else {
                    p = (r + t) % (ne - 1);
                    q = (r - t + (ne - 1)) % (ne - 1);
                }
                double c = 1.0, s = 0.0;
                zd ph = zmk(1.0, 0.0);
                if (p < n && q < n) {
                    const zd apq = A[p + (size_t)q * n];
                    const double rr = hypot(apq.x, apq.y);
                    const double app = A[p + (size_t)p * n].x, aqq = A[q + (size_t)q * n].x;
                    if (rr > 1e-300 && rr > 1e-18 * sqrt(fabs(app * aqq))) {
                        const double tau = (aqq - app) / (2.0 * rr);
                        const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + tt * tt);
                        s = tt * c;
                        ph = zmk(apq.x / rr, apq.y / rr);
                    }
                }
                sp[t] = p;
                sq[t] = q;
                sc[t] = c;
                sv[t] = s;
                sph[t] = ph;
            }
            __syncthreads();
            // columns: A <- A G, V <- V G
            for (int e = tid; e < n * np; e += nt) {
                const int i = e % n, t = e / n;
                const int p = sp[t], q = sq[t];
                if (p >= n || q >= n || sv[t] == 0.0) continue;
                const double c = sc[t], s = sv[t];
                const zd em = zconj(sph[t]);  // e^{-i phi}
                zd* ap = A + i + (size_t)p * n;
                zd* aq = A + i + (size_t)q * n;
                const zd xp = *ap, xq = zmul(em, *aq);
                *ap = zsub(zscale(xp, c), zscale(xq, s));
                *aq = zadd(zscale(xp, s), zscale(xq, c));
                zd* vp = V + i + (size_t)p * n;
                zd* vq = V + i + (size_t)q * n;
                const zd yp = *vp, yq = zmul(em, *vq);
                *vp = zsub(zscale(yp, c), zscale(yq, s));
                *vq = zadd(zscale(yp, s), zscale(yq, c));
            }
            __syncthreads();
            // rows: A <- G^H A
            for (int e = tid; e < n * np; e += nt) {
                const int j = e % n, t = e / n;
                const int p = sp[t], q = sq[t];
                if (p >= n || q >= n || sv[t] == 0.0) continue;
                const double c = sc[t], s = sv[t];
                const zd ep = sph[t];  // e^{i phi}
                zd* ap = A + p + (size_t)j * n;
                zd* aq = A + q + (size_t)j * n;
                const zd xp = *ap, xq = zmul(ep, *aq);
                *ap = zsub(zscale(xp, c), zscale(xq, s));
                *aq = zadd(zscale(xp, s), zscale(xq, c));
            }
            __syncthreads();
            for (int t = tid; t < np; t += nt) {
                const int p = sp[t], q = sq[t];
                if (p >= n || q >= n || sv[t] == 0.0) continue;
                A[p + (size_t)q * n] = zmk(0.0, 0.0);
                A[q + (size_t)p * n] = zmk(0.0, 0.0);
                A[p + (size_t)p * n].y = 0.0;
                A[q + (size_t)q * n].y = 0.0;
            }
            __syncthreads();
        }
    }
    if (!conv && tid == 0) atomicOr(flag, 1);
    // ascending order: rank by counting (ties by index), then permute the
    // columns of V through A, which is no longer needed
    __syncthreads();
    for (int i = tid; i < n; i += nt) {
        const double di = A[i + (size_t)i * n].x;
        int rk = 0;
        for (int j = 0; j < n; ++j) {
            const double dj = A[j + (size_t)j * n].x;
            rk += (dj < di) || (dj == di && j < i);
        }
        w[rk] = di;
        if (i < 512) sp[i] = rk; else sq[i - 512] = rk;
    }
    __syncthreads();
    for (size_t e = tid; e < nn; e += nt) {
        const int i = (int)(e % n), j = (int)(e / n);
        const int rk = (j < 512) ? sp[j] : sq[j - 512];
        A[i + (size_t)rk * n] = V[e];
    }
    __syncthreads();
    for (size_t e = tid; e < nn; e += nt) V[e] = A[e];
}

int launch_jacobi(zd* const* mats, double* const* vals, zd* const* vecs, int nbatch, int n,
                  int max_sweeps, int* d_flag, cudaStream_t s) {
    if (n > 1024) return -1;
    k_jacobi<<<nbatch, 1024, 0, s>>>(mats, vals, vecs, n, max_sweeps, d_flag);
    return 0;
}

// wtmp[i, n] *= e^{-i dt lambda_i}
__global__ void k_eigphase(StepArgs a) {
    const KDev& K = a.kd[blockIdx.z];
    const int e = blockIdx.x * 256 + threadIdx.x;
    if (e >= a.naux * a.ns) return;
    const int i = e % a.naux;
    const double ph = -a.dt * K.eval[i];
    K.wtmp[e] = zmul(zmk(cos(ph), sin(ph)), K.wtmp[e]);
}

// column j of each matrix scaled by 1/sqrt(vals[j]) (mode 0)
__global__ void k_scale_cols(zd* const* mats, const double* const* vals, int n, int mode) {
    zd* M = mats[blockIdx.z];
    const double* v = vals[blockIdx.z];
    const int e = blockIdx.x * 256 + threadIdx.x;
    if (e >= n * n) return;
    const int j = e / n;
    double f = 1.0;
    if (mode == 0) f = 1.0 / sqrt(v[j]);
    M[e] = zscale(M[e], f);
}
void launch_scale_cols(zd* const* mats, const double* const* vals, int nbatch, int n, int mode,
                       cudaStream_t s) {
    dim3 grid((n * n + 255) / 256, 1, nbatch);
    k_scale_cols<<<grid, 256, 0, s>>>(mats, vals, n, mode);
}

// Scale column i of CC (and of an optional companion matrix) so that the
// sum of its coefficients is real and positive.
__global__ void __launch_bounds__(256) k_phase_fix(const KDev* kd, int naux, zd* const* extra,
                                                   const int* ldextra, int nextra_rows) {
    __shared__ double sh[32];
    const int k = blockIdx.z, i = blockIdx.x;
    const KDev& K = kd[k];
    zd* col = K.caux + (size_t)i * K.nb;
    double sr = 0.0, si = 0.0;
    for (int r = threadIdx.x; r < K.nb; r += blockDim.x) {
        sr += col[r].x;
        si += col[r].y;
    }
    sr = block_sum(sr, sh);
    si = block_sum(si, sh);
    const double m = hypot(sr, si);
    const zd ph = (m > 0.0) ? zmk(sr / m, -si / m) : zmk(1.0, 0.0);
    for (int r = threadIdx.x; r < K.nb; r += blockDim.x) col[r] = zmul(col[r], ph);
    if (extra) {
        zd* x = extra[k] + (size_t)i * ldextra[k];
        for (int r = threadIdx.x; r < nextra_rows; r += blockDim.x) x[r] = zmul(x[r], ph);
    }
}
void launch_phase_fix(const KDev* kd, int nk, int naux, zd* const* extra, const int* ldextra,
                      int nextra_rows, cudaStream_t s) {
    dim3 grid(naux, 1, nk);
    k_phase_fix<<<grid, 256, 0, s>>>(kd, naux, extra, ldextra, nextra_rows);
}

// ------------------------------------------------------------ orchestration
// the cooperative series forms its own rows of HH when each block owns one
// row and the row fits the registers of the block's threads
int cheb_direct(const StepArgs& a) {
    return (a.coop_grid >= a.nk * a.naux && a.naux <= CHEB_JU * CHEB_THREADS && a.ns <= 4) ? 1 : 0;
}
// per-row state of the cooperative series: 3 ns complex per row of a block
static size_t cheb_coop_smem(const StepArgs& a, int grid) {
    const int nrow = a.nk * a.naux;
    const int rows = grid > 0 ? (nrow + grid - 1) / grid : 0;
    return (size_t)rows * 3 * a.ns * sizeof(zd);
}
static cudaError_t launch_cheb_coop_raw(const StepArgs& a, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.coop_grid);
    cfg.blockDim = dim3(a.cheb_tile ? CT_THREADS : CHEB_THREADS);
    cfg.dynamicSmemBytes = a.cheb_tile ? cheb_tile_smem(a.naux) : cheb_coop_smem(a, a.coop_grid);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (a.cheb_tile) return cudaLaunchKernelEx(&cfg, k_cheb_tile, a);
    const int direct = cheb_direct(a);
    if (a.ns <= 2) return cudaLaunchKernelEx(&cfg, k_cheb_coop<2>, a, direct);
    if (a.ns <= 4) return cudaLaunchKernelEx(&cfg, k_cheb_coop<4>, a, direct);
    return cudaLaunchKernelEx(&cfg, k_cheb_coop<8>, a, direct);
}
void launch_cheb_coop(const StepArgs& a, cudaStream_t s) { launch_cheb_coop_raw(a, s); }

// Blocks for the cooperative series: all must be resident at once (the
// launch guarantees it or fails), and the launch must be capturable in a
// graph on this driver; otherwise 0 (one launch per term).
// The tile form of the series for 4 < N_s <= 64 when one tile per block fits
// on the GPU at once: its grid, or 0.
// It pays when the columns fill most lanes and the tiles cover the GPU (mos2_16k,
// N_s 60 on 16 x 38 tiles: 8.3 ms against 15.0 ms per series; co_12000, N_s 7 on
// 50 tiles: 3.0 ms against 0.22 ms).  RTTDDFT_CHEB_TILE=1 or =0 in the
// environment forces the choice (the tests run both forms).
static int prepare_cheb_tile(const StepArgs& a0, int nsm) {
    if (a0.ns <= 4 || a0.ns > CT_COLS) return 0;
    const int grid = a0.nk * ((a0.naux + CT_ROWS - 1) / CT_ROWS);
    const char* force = getenv("RTTDDFT_CHEB_TILE");
    const bool forced = force && force[0] == '1' && force[1] == 0;
    if (force && force[0] == '0' && force[1] == 0) return 0;
    if (!forced && (a0.ns < CT_COLS / 2 || grid < nsm)) return 0;
    const size_t smem = cheb_tile_smem(a0.naux);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_cheb_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cheb_tile, CT_THREADS, smem) != cudaSuccess ||
        per_sm <= 0 || grid > per_sm * nsm) {
        cudaGetLastError();
        return 0;
    }
    return grid;
}

int prepare_cheb_coop(const StepArgs& a0, cudaStream_t s, int* tile) {
    int dev = 0, coop = 0, nsm = 0, per_sm = 0;
    *tile = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (!coop || nsm <= 0) return 0;
    if (const int gt = prepare_cheb_tile(a0, nsm)) {
        StepArgs a = a0;
        a.coop_grid = gt;
        a.cheb_tile = 1;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            cudaError_t e1 = launch_cheb_coop_raw(a, s);
            cudaError_t e2 = cudaStreamEndCapture(s, &g);
            int ok = (e1 == cudaSuccess && e2 == cudaSuccess && g != nullptr);
            if (ok) {
                cudaGraphExec_t x = nullptr;
                ok = cudaGraphInstantiate(&x, g, 0) == cudaSuccess;
                if (x) cudaGraphExecDestroy(x);
            }
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            if (ok) {
                *tile = 1;
                return gt;
            }
        } else {
            cudaGetLastError();
        }
    }
    // one block per row while the rows last, at most four blocks per SM
    // (more blocks would lengthen the barrier's arrival chain)
    const int nrow = a0.nk * a0.naux;
    int grid = nrow < 4 * nsm ? nrow : 4 * nsm;
    const size_t smem = cheb_coop_smem(a0, grid);
    const void* fn = a0.ns <= 2 ? (const void*)k_cheb_coop<2>
                                : (a0.ns <= 4 ? (const void*)k_cheb_coop<4> : (const void*)k_cheb_coop<8>);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, CHEB_THREADS, smem);
    if (e != cudaSuccess || per_sm <= 0 || grid > per_sm * nsm) {
        cudaGetLastError();
        return 0;
    }
    StepArgs a = a0;
    a.coop_grid = grid;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaError_t e1 = launch_cheb_coop_raw(a, s);
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    int ok = (e1 == cudaSuccess && e2 == cudaSuccess && g != nullptr);
    if (ok) {
        cudaGraphExec_t x = nullptr;
        ok = cudaGraphInstantiate(&x, g, 0) == cudaSuccess;
        if (x) cudaGraphExecDestroy(x);
    }
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return ok ? grid : 0;
}

void launch_set_cur(const StepArgs& a, cudaStream_t s) { k_set_cur<<<1, 1, 0, s>>>(a); }

void launch_prep_coef(const StepArgs& a, cudaStream_t s) {
    if (a.prop == 1) return;
    k_coef<<<a.nk, 32, 0, s>>>(a);
}

void launch_subspace_current(const StepArgs& a, int set_gs, cudaStream_t s) {
    launch_post(a, 0, 1, s);
    launch_finalize(a, set_gs, s);
}

static inline void mark(TraceHook* tr, const char* name, cudaStream_t s) {
    if (!tr || tr->n >= tr->cap) return;
    tr->names[tr->n] = name;
    cudaEventRecordWithFlags(tr->ev[tr->n], s, cudaEventRecordExternal);
    tr->n += 1;
}

template <int NT>
static size_t toep_smem(const StepArgs& a, size_t tc, size_t tt) {
    const size_t t = (size_t)BT * NT * tc + (size_t)BT * sizeof(int) + (size_t)a.wmax * tt;
    const size_t b = (size_t)a.msegw * 2 * NT * tc;
    return t > b ? t : b;
}

template <typename TA, typename TT, typename TC, int NT>
static int back_launch(const StepArgs& a, int maxng, cudaStream_t s, TraceHook* tr, cudaEvent_t join) {
    // in the tensor-core form the interstitial slots are done already: only
    // the back-projection slots run here, and they need no table window
    const int slot0 = a.ith ? a.nseg : 0;
    const size_t sm = slot0 ? (size_t)a.msegw * 2 * NT * sizeof(TC) : toep_smem<NT>(a, sizeof(TC), sizeof(TT));
    // with the back-projection on the tensor cores too, no slot kernel runs
    dim3 gt((maxng + BT - 1) / BT, a.tcback ? 0 : a.nslot - slot0, a.nk);
    dim3 gb((maxng + BKB - 1) / BKB, 1, a.nk);
    int nl = 0;
    if (gt.y == 0) {
        // both parts arrive whole (K.th and K.tb): every column in one launch
        if (join) cudaStreamWaitEvent(s, join, 0);
        k_back<NT><<<gb, BKB, 0, s>>>(a, 0, a.ns);
        mark(tr, "back_finish", s);
        return 1;
    }
    for (int n0 = 0; n0 < a.ns; n0 += NT) {
        ++nl;
        k_toep_seg<TA, TT, TC, NT><<<gt, BT, sm, s>>>(a, n0, slot0);
        mark(tr, slot0 ? "backprojection" : "toeplitz_and_backprojection", s);
        if (join && n0 == 0) cudaStreamWaitEvent(s, join, 0);  // the interstitial rows of the side stream
        k_back<NT><<<gb, BKB, 0, s>>>(a, n0, std::min(n0 + NT, a.ns));
        mark(tr, "back_finish", s);
        ++nl;
    }
    return nl;
}

// Opt the slot kernels in to the shared memory their table window needs.
// The attribute is global per kernel, so it only ever grows (a context with
// a smaller window must not lower another context's limit).
static size_t g_toep_smem[6];
static size_t g_locw_smem[3];
int prepare_back_kernels(const StepArgs& a) {
    cudaError_t e = cudaSuccess;
    if (a.prec >= 1 && a.ns > LOCW_MIN_NS && a.at_n > 0) {
        // the wide muffin-tin kernel stages [Q; C_lo] of one atom (FP32)
        const size_t need = (size_t)a.at_maxm * a.ns * sizeof(zf);
        const int w = a.ns <= 32 ? 0 : (a.ns <= 64 ? 1 : 2);
        if (need > g_locw_smem[w]) {
            e = w == 0 ? cudaFuncSetAttribute(k_local_wide<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need)
                : w == 1 ? cudaFuncSetAttribute(k_local_wide<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need)
                         : cudaFuncSetAttribute(k_local_wide<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
            if (e != cudaSuccess) return 1;
            g_locw_smem[w] = need;
        }
    }
    int slot = 0;
#define RTD_SET(TA, TT, TC, NT)                                                                      \
    {                                                                                                \
        const size_t need = toep_smem<NT>(a, sizeof(TC), sizeof(TT));                                \
        if (need > g_toep_smem[slot]) {                                                              \
            e = cudaFuncSetAttribute(k_toep_seg<TA, TT, TC, NT>,                                     \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);         \
            if (e != cudaSuccess) return (int)e;                                                     \
            g_toep_smem[slot] = need;                                                                \
        }                                                                                            \
        ++slot;                                                                                      \
    }
    // only the instances of the context's form (FP64 entries, or FP32 ones)
    if (a.prec == 0) {
        RTD_SET(zd, zd, zd, 2) RTD_SET(zd, zd, zd, 4) RTD_SET(zd, zd, zd, 8)
    } else {
        slot = 3;
        RTD_SET(zf, zf, zf, 2) RTD_SET(zf, zf, zf, 4) RTD_SET(zf, zf, zf, 8)
    }
#undef RTD_SET
    return 0;
}

int launch_operator_pass(const StepArgs& a, const StepPlan& p, cudaStream_t s, TraceHook* tr) {
    const bool f32 = a.prec >= 1;
    int nl = 0;
    // trace mode keeps one stream so that its events time every launch in turn
    const bool fork = p.fft && p.side && !tr;
    const cudaEvent_t join = fork ? p.ev_join : nullptr;
    if (p.fft) {
        // V~ * C_G by FFT (th), the current table V~ + s dV~ when the change is on.
        // It needs only C, so it runs on the side stream beside the matching
        // rows, the muffin-tin blocks and the back-projection, and k_back waits for it.
        cudaStream_t fs = s;
        if (fork) {
            cudaEventRecord(p.ev_fork, s);
            cudaStreamWaitEvent(p.side, p.ev_fork, 0);
            fs = p.side;
        }
        nl += launch_fft_conv(p.fft, p.td_op, a.kofs, a.nk, a.ns, 0, a.dv_on, &a.st->cur_s, fs);
        if (fork) cudaEventRecord(p.ev_join, p.side);
        mark(tr, "fft_interstitial", fs);
    }
    if (a.prec >= 2) {
        // tensor cores: V~ * C_G (unless the FFT route gives it) and Q = A C_G in
        // split-BF16 launches
        launch_tc_pack(p.tc, a, s);
        mark(tr, "tc_pack_c", s);
        nl += launch_tc_operator(p.tc, a, s, p.fft != nullptr);
        mark(tr, p.fft ? "tc_forward" : "tc_interstitial_and_forward", s);
        launch_tc_reduce(p.tc, a, s, p.fft != nullptr);
        mark(tr, "tc_reduce", s);
        nl += 2;
    } else {
        if (a.toep_global && !p.fft) {
            // a table window too large for shared memory: V~ * C_G (V~ + s dV~ when the
            // change is on) with the table gathered through L1/L2, FP64, into K.th
            launch_toeplitz(a.kd, p.td_op + a.kofs, a.nk, p.maxng, a.ns, a.dv_on ? a.vstep : a.vtab, a.vt_center, 0,
                            0, nullptr, s);
            mark(tr, "toeplitz_global", s);
            ++nl;
        }
        if (a.ma > 0) {
            // Q = A C_G = (A^H)^H C_G: one warp per matching row; split-K in FP64
            const bool summed = launch_gemm_cn(p.gd_fwd, a.nk, a.ma, p.maxng, a.ns, p.kc_fwd, p.part, 0, f32,
                                               nullptr, s, p.tile_cnt);
            mark(tr, "gemm_forward", s);
            ++nl;
            if (!summed) {
                launch_split_reduce(p.gd_fwd, a.nk, a.ma, a.ns, p.kc_fwd, p.part, 0, s);
                mark(tr, "split_reduce_forward", s);
                ++nl;
            }
        }
    }
    if (a.lrows > 0 && f32 && p.gd_mt1 && a.mtg) {
        nl += launch_mt_gemm(a, p, s);
        mark(tr, "local_mt", s);
    } else if (a.lrows > 0) {
        ++nl;
        dim3 g(a.lrows, 1, a.nk);
        if (f32 && a.ns > LOCW_MIN_NS) {
            // lanes own columns; row chunks per atom so that about two blocks per SM work
            const size_t sm = (size_t)a.at_maxm * a.ns * sizeof(zf);
            int rc = std::max(4, (2 * 152 + a.at_n * a.nk - 1) / (a.at_n * a.nk));
            rc = std::min(rc, std::max(1, a.at_maxm / 4));
            dim3 gw(a.at_n * rc, 1, a.nk);
            if (a.ns <= 32) k_local_wide<1><<<gw, 128, sm, s>>>(a, rc);
            else if (a.ns <= 64) k_local_wide<2><<<gw, 128, sm, s>>>(a, rc);
            else k_local_wide<4><<<gw, 128, sm, s>>>(a, rc);
        } else if (f32) {
            if (a.ns <= 2) k_local<zf, 2><<<g, 32, 0, s>>>(a);
            else k_local<zf, 4><<<g, 32, 0, s>>>(a);
        } else {
            if (a.ns <= 2) k_local<zd, 2><<<g, 32, 0, s>>>(a);
            else k_local<zd, 4><<<g, 32, 0, s>>>(a);
        }
        mark(tr, "local_mt", s);
    }
    if (a.tcback) {
        // A^H [hQ | oQ] on the tensor cores
        nl += launch_tc_back(p.tc, a, s);
        mark(tr, "tc_backprojection", s);
    }
    if (f32) {
        if (a.ns <= 2) nl += back_launch<zf, zf, zf, 2>(a, p.maxng, s, tr, join);
        else if (a.ns <= 4) nl += back_launch<zf, zf, zf, 4>(a, p.maxng, s, tr, join);
        else nl += back_launch<zf, zf, zf, 8>(a, p.maxng, s, tr, join);
    } else {
        if (a.ns <= 2) nl += back_launch<zd, zd, zd, 2>(a, p.maxng, s, tr, join);
        else if (a.ns <= 4) nl += back_launch<zd, zd, zd, 4>(a, p.maxng, s, tr, join);
        else nl += back_launch<zd, zd, zd, 8>(a, p.maxng, s, tr, join);
    }
    return nl;
}

// Eq. v_MT and Eq. v_interstitial rebuilt from the scaled blocks:
// dVV = L^H (s dh) L + CC_G^H (s dV~ * CC_G).  In the tensor-core forms the
// interstitial convolution runs on tcgen05 (split-BF16) and its projection in
// FP32; otherwise both in FP64.  Returns the launches.
static int launch_dv_rebuild(const StepArgs& a, const StepPlan& p, cudaStream_t s, TraceHook* tr) {
    if (a.hartree) {
        // dVV = [sum_a L^H dh_a L] + CC_G^H (dV~ * CC_G) with dV~ (and dh, when the
        // muffin-tin part is on) from the previous step's density
        int nl = 0, beta = 0;
        if (a.mt_u != 0.0 && p.gd_dvw) {
            const bool mt32 = a.prec >= 1 && p.gd_dvw32 && p.gd_dvg32;
            launch_gemm_nn(mt32 ? p.gd_dvw32 : p.gd_dvw, p.n_dvw, p.maxm, p.maxm, a.naux, 0, nullptr, 0, mt32,
                           &a.st->cur_s, s);
            launch_gemm_cn(mt32 ? p.gd_dvg32 : p.gd_dvg, a.nk, a.naux, a.lrows, a.naux, 0, nullptr, 0, mt32, nullptr,
                           s);
            mark(tr, "hartree_mt_blocks", s);
            nl += 2;
            beta = 1;
        }
        launch_fft_conv(p.fft, p.td_dv, a.kofs, a.nk, a.naux, 1, 1, &a.st->cur_s, s);
        mark(tr, "hartree_interstitial_fft", s);
        if (p.gd_dvi32) {
            // FP32 form: CC_G^H T streaming the FP32 copy of CC, FP64 sums of the K slices
            launch_gemm_cn(p.gd_dvi32, a.nk, a.naux, p.maxng, a.naux, p.kc_dvi, p.part_dv, 0, true, nullptr, s);
            launch_split_reduce(p.gd_dvi32, a.nk, a.naux, a.naux, p.kc_dvi, p.part_dv, beta, s);
            mark(tr, "hartree_project", s);
            return nl + 1;
        }
        launch_gemm_cn(p.gd_dvi, a.nk, a.naux, p.maxng, a.naux, 0, nullptr, beta, false, nullptr, s);
        mark(tr, "hartree_project", s);
        return nl;  // the FFT launches are counted by the caller
    }
    // the muffin-tin four blocks: FP32 in the reduced-precision forms, FP64 otherwise
    const bool mt32 = a.prec >= 1 && p.gd_dvw32 && p.gd_dvg32;
    launch_gemm_nn(mt32 ? p.gd_dvw32 : p.gd_dvw, p.n_dvw, p.maxm, p.maxm, a.naux, 0, nullptr, 0, mt32,
                   &a.st->cur_s, s);
    mark(tr, "dv_mt_blocks", s);
    launch_gemm_cn(mt32 ? p.gd_dvg32 : p.gd_dvg, a.nk, a.naux, a.lrows, a.naux, 0, nullptr, 0, mt32, nullptr, s);
    mark(tr, "dv_mt_project", s);
    if (a.prec >= 2 && p.tc && !p.fft && tc_dv_ready(p.tc) && p.gd_dvi32) {
        launch_tc_dv_toeplitz(p.tc, a, p.td_dv, s);
        mark(tr, "tc_dv_interstitial", s);
        launch_gemm_cn(p.gd_dvi32, a.nk, a.naux, p.maxng, a.naux, p.kc_dvi, p.part_dv, 0, true, nullptr, s);
        launch_split_reduce(p.gd_dvi32, a.nk, a.naux, a.naux, p.kc_dvi, p.part_dv, 1, s);
        mark(tr, "dv_interstitial_project", s);
        return 4 + 2 * tc_dv_tiles(p.tc);
    }
    int nl = 3;
    if (p.fft) {
        // T = s (dV~ * CC_G) by FFT over the N_aux columns
        nl += launch_fft_conv(p.fft, p.td_dv, a.kofs, a.nk, a.naux, 1, 1, &a.st->cur_s, s);
        mark(tr, "dv_interstitial_fft", s);
    } else {
        launch_toeplitz(a.kd, p.td_dv, a.nk, p.maxng, a.naux, a.dvtab, a.vt_center, 0, 0, &a.st->cur_s, s);
        mark(tr, "dv_interstitial_toeplitz", s);
        ++nl;
    }
    if (a.prec >= 1 && p.gd_dvi32) {
        // reduced-precision forms: CC_G^H T from the FP32 copy of CC, FP64 sums of the K slices
        launch_gemm_cn(p.gd_dvi32, a.nk, a.naux, p.maxng, a.naux, p.kc_dvi, p.part_dv, 0, true, nullptr, s);
        launch_split_reduce(p.gd_dvi32, a.nk, a.naux, a.naux, p.kc_dvi, p.part_dv, 1, s);
        ++nl;
    } else {
        launch_gemm_cn(p.gd_dvi, a.nk, a.naux, p.maxng, a.naux, 0, nullptr, 1, false, nullptr, s);
    }
    mark(tr, "dv_interstitial_project", s);
    return nl;
}

void launch_step(const StepArgs& a, const StepPlan& p, cudaStream_t s, int* nlaunch, TraceHook* tr) {
    int nl = 0;
    const bool f32 = a.prec >= 1;
    const int nn = a.naux * a.naux;
    if (a.dv_on) {
        k_set_cur<<<1, 1, 0, s>>>(a);
        mark(tr, "set_cur", s);
        ++nl;
        if (a.hartree) {
            nl += launch_dv_rebuild(a, p, s, tr) + (p.fft_launches > 0 ? p.fft_launches : 5) + 1;
        } else {
            // Eq. v_MT and Eq. v_interstitial rebuilt from the scaled blocks:
            // dVV = L^H (s dh) L + CC_G^H (s dV~ * CC_G)
            k_vstep<<<(a.nvt + 255) / 256, 256, 0, s>>>(a);
            mark(tr, "dv_table", s);
            nl += 1 + launch_dv_rebuild(a, p, s, tr);
        }
    }
    if (!(a.prop != 1 && a.coop_grid > 0 && cheb_direct(a))) {
        k_hsub<<<dim3((nn + 255) / 256, 1, a.nk), 256, 0, s>>>(a);
        mark(tr, "hsub", s);
        ++nl;
    }
    if (a.prop == 1) {
        launch_jacobi(p.jac_mats, p.jac_vals, p.jac_vecs, a.nk, a.naux, p.max_sweeps, p.d_flag, s);
        mark(tr, "jacobi", s);
        launch_gemm_cn(p.gd_evh, a.nk, a.naux, a.naux, a.ns, 0, nullptr, 0, false, nullptr, s);
        k_eigphase<<<dim3((a.naux * a.ns + 255) / 256, 1, a.nk), 256, 0, s>>>(a);
        launch_gemm_nn(p.gd_evn, a.nk, a.naux, a.naux, a.ns, 0, nullptr, 0, false, nullptr, s);
        mark(tr, "eig_apply", s);
        nl += 4;
    } else if (a.coop_grid > 0) {
        launch_cheb_coop(a, s);
        mark(tr, "chebyshev_series", s);
        ++nl;
    } else {
        dim3 g(a.naux, 1, a.nk);
        for (int t = 1; t < a.nterms; ++t) {
            const int last = (t == a.nterms - 1);
            if (a.ns <= 2) k_cheb<2><<<g, 128, 0, s>>>(a, t, last);
            else if (a.ns <= 4) k_cheb<4><<<g, 128, 0, s>>>(a, t, last);
            else k_cheb<8><<<g, 128, 0, s>>>(a, t, last);
            mark(tr, "chebyshev_term", s);
            ++nl;
        }
    }
    // C = CC theta (Eq. approximation_coefficients)
    if (p.tcc) {
        nl += launch_tcc_expand(p.tcc, a, s);
        mark(tr, "gemm_expand", s);
    } else {
        launch_gemm_nn(p.gd_expand, a.nk, p.maxnb, a.naux, a.ns, p.kc_expand, p.kc_expand > 0 ? p.part : nullptr,
                       0, f32, nullptr, s);
        mark(tr, "gemm_expand", s);
        ++nl;
    }
    if (!p.tcc && p.kc_expand > 0) {
        launch_split_reduce(p.gd_expand, a.nk, p.maxnb, a.ns, p.kc_expand, p.part, 0, s);
        mark(tr, "split_reduce_expand", s);
        ++nl;
    }
    nl += launch_operator_pass(a, p, s, tr);
    // theta~ = CC^H (S C): split-K partials, finished per row in k_post
    if (p.tcc) nl += launch_tcc_project(p.tcc, a, p.part, s) - 1;
    else launch_gemm_cn(p.gd_proj, a.nk, a.naux, p.maxnb, a.ns, p.kc_proj, p.part, 0, f32, nullptr, s);
    mark(tr, "gemm_project", s);
    launch_post(a, 1, a.reproject ? 0 : 1, s);
    mark(tr, "project_finish_current", s);
    if (!a.reproject && a.ns > JRHO_MIN_NS) ++nl;
    if (a.ns > 4) {
        k_gram_dev<<<dim3(a.ns, a.nk), 256, 0, s>>>(a);
        mark(tr, "gram", s);
        ++nl;
    }
    nl += 2;
    if (a.reproject) {
        launch_gemm_cn(p.gd_g2, a.nk, a.ns, a.naux, a.ns, 0, nullptr, 0, false, nullptr, s);
        k_reproj<<<dim3((a.naux * a.ns + 255) / 256, 1, a.nk), 256, 0, s>>>(a);
        launch_post(a, 0, 1, s);
        mark(tr, "reproject", s);
        nl += 3;
    }
    launch_finalize(a, 0, s);
    mark(tr, "finalize", s);
    nl += 2;
    if (a.hartree) {
        // the density of C_{k+1} sets the potential change of the next step
        if (p.gd_exp64) {
            launch_gemm_nn(p.gd_exp64, a.nk, p.maxnb, a.naux, a.ns, 0, nullptr, 0, false, nullptr, s);
            ++nl;
        }
        if (a.mt_u != 0.0 && p.gd_mty) nl += launch_mt_feedback(a, p, 0, fft_l1(p.fft), s);
        nl += launch_fft_hartree(p.fft, p.td_dens, a.nk, a.ns, a.occ, a.wk, a.flag, s);
        mark(tr, "hartree_density_poisson", s);
    }
    if (nlaunch) *nlaunch = nl;
}

void launch_vstep(const StepArgs& a, cudaStream_t s) { k_vstep<<<(a.nvt + 255) / 256, 256, 0, s>>>(a); }

// Raise flag bit 2 if a device-resident sample exceeds the declared bounds.
__global__ void k_check_samples(const double* a, int na, double amax, const double* s, int ns,
                                double smax, int* flag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < na || i < ns; i += gridDim.x * blockDim.x) {
        if (i < na) {
            const double* q = a + 3 * (size_t)i;
            const double m = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
            if (!(m <= amax)) atomicOr(flag, 2);
        }
        if (i < ns && !(fabs(s[i]) <= smax)) atomicOr(flag, 2);
    }
}
void launch_check_samples(const double* a, int na, double amax, const double* s, int ns, double smax,
                          int* flag, cudaStream_t st) {
    const int n = na > ns ? na : ns;
    if (n == 0) return;
    k_check_samples<<<(n + 255) / 256 < 64 ? (n + 255) / 256 : 64, 256, 0, st>>>(a, na, amax, s, ns, smax, flag);
}

__global__ void k_set_cstep(DevState* st, int c) { st->cstep = c; }

// The subspace part of a step only (HH(t_k) and its Chebyshev series, one
// launch per term): what the adjoint recomputes.  cstep selects the sample.
void launch_propagate_only(const StepArgs& a, const StepPlan& p, int cstep, cudaStream_t s) {
    k_set_cstep<<<1, 1, 0, s>>>(a.st, cstep);
    if (a.dv_on) {
        k_set_cur<<<1, 1, 0, s>>>(a);
        k_vstep<<<(a.nvt + 255) / 256, 256, 0, s>>>(a);
        launch_dv_rebuild(a, p, s, nullptr);
    }
    k_hsub<<<dim3((a.naux * a.naux + 255) / 256, 1, a.nk), 256, 0, s>>>(a);
    dim3 g(a.naux, 1, a.nk);
    for (int t = 1; t < a.nterms; ++t) {
        const int last = (t == a.nterms - 1);
        if (a.ns <= 2) k_cheb<2><<<g, 128, 0, s>>>(a, t, last);
        else if (a.ns <= 4) k_cheb<4><<<g, 128, 0, s>>>(a, t, last);
        else k_cheb<8><<<g, 128, 0, s>>>(a, t, last);
    }
}

// HH(t_k) only (the adjoint's reverse sweep needs the matrix of step cstep)
void launch_hsub_only(const StepArgs& a, const StepPlan& p, int cstep, cudaStream_t s) {
    k_set_cstep<<<1, 1, 0, s>>>(a.st, cstep);
    if (a.dv_on) {
        k_set_cur<<<1, 1, 0, s>>>(a);
        launch_dv_rebuild(a, p, s, nullptr);
    }
    k_hsub<<<dim3((a.naux * a.naux + 255) / 256, 1, a.nk), 256, 0, s>>>(a);
}

// J contributions of the current theta (rows into part_post[.][1..3])
void launch_subspace_j(const StepArgs& a, cudaStream_t s) { launch_post(a, 0, 1, s); }

// ------------------------------------------------------------ muffin-tin density feedback
// Per atom the density matrix of its matching and local-orbital channels,
// n_a = sum_k w_k sum_j f_j y_kaj y_kaj^H with y = the atom's rows of the
// state's local coordinates L theta (FP64: L = E_a CC from set-up, theta the
// FP64 state), one thread per entry (i, j) of the atom's m x m block.
// reference: store n_a as n0; otherwise dh_a = U (n_a - n0_a) (and its FP32
// copy), with sum |dh_a|^2 per atom added to mt_fn2 for the bound.
__global__ void k_mt_density(StepArgs a, int reference) {
    __shared__ double red[8];
    const AtomTab& at = *a.at;
    const int al = blockIdx.y;
    if (al >= at.n) return;
    const int m = at.m[al], lr = a.lrows, ns = a.ns;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    double sq = 0.0;
    if (e < m * m) {
        const int i = e % m, j = e / m;
        const int ri = at.loff[al] + i, rj = at.loff[al] + j;
        double re = 0.0, im = 0.0;
        for (int k = 0; k < a.nk; ++k) {
            const zd* Y = a.mty + (size_t)k * lr * ns;
            double kr = 0.0, ki = 0.0;
            for (int c = 0; c < ns; ++c) {
                const zd yi = Y[ri + (size_t)c * lr], yj = Y[rj + (size_t)c * lr];
                const double f = a.occ[c];
                kr += f * (yi.x * yj.x + yi.y * yj.y);  // yi conj(yj)
                ki += f * (yi.y * yj.x - yi.x * yj.y);
            }
            re += a.wk[k] * kr;
            im += a.wk[k] * ki;
        }
        const size_t idx = at.boff[al] + i + (size_t)j * m;
        if (reference) {
            ((zd*)a.mtn0)[idx] = zmk(re, im);
        } else {
            const zd n0 = a.mtn0[idx];
            const zd d = zmk(a.mt_u * (re - n0.x), a.mt_u * (im - n0.y));
            ((zd*)a.dh)[idx] = d;
            if (a.dh32) a.dh32[idx] = tof(d);
            sq = d.x * d.x + d.y * d.y;
        }
    }
    if (reference) return;
    sq = warp_sum(sq);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(a.mt_fn2 + al, t);  // only compared with a bound: the order does not matter
    }
}
// sum_a ||dh_a||_F max_k ||L_ka||_F^2 >= ||sum_a L_ka^H dh_a L_ka||_2 added to the
// accumulator that the step compares with the Chebyshev interval's bound
__global__ void k_mt_bound(StepArgs a, double* l1) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double b = 0.0;
    for (int al = 0; al < a.at->n; ++al) {
        b += sqrt(a.mt_fn2[al]) * a.mt_lnorm[al];
        a.mt_fn2[al] = 0.0;
    }
    *l1 += b;
}
// per atom max_k ||L_ka||_F^2 (set-up), as the integer maximum of non-negative doubles
__global__ void k_mt_lnorm(StepArgs a) {
    __shared__ double red[8];
    const AtomTab& at = *a.at;
    const int al = blockIdx.y, k = blockIdx.z;
    if (al >= at.n) return;
    const KDev& K = a.kd[k];
    const int m = at.m[al], n = a.naux;
    double sq = 0.0;
    for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
        const zd v = K.lloc[at.loff[al] + e % m + (size_t)(e / m) * a.lrows];
        sq += v.x * v.x + v.y * v.y;
    }
    sq = warp_sum(sq);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicMax((unsigned long long*)(a.mt_lnorm + al), (unsigned long long)__double_as_longlong(t));
    }
}

int launch_mt_feedback(const StepArgs& a, const StepPlan& p, int reference, double* l1, cudaStream_t s) {
    // the state's local coordinates L theta (FP64, every k)
    launch_gemm_nn(p.gd_mty, a.nk, a.lrows, a.naux, a.ns, 0, nullptr, 0, false, nullptr, s);
    const int mm = a.at_maxm * a.at_maxm;
    k_mt_density<<<dim3((mm + 255) / 256, a.at_n), 256, 0, s>>>(a, reference);
    if (reference) return 2;
    k_mt_bound<<<1, 32, 0, s>>>(a, l1);
    return 3;
}
void launch_mt_lnorm(const StepArgs& a, cudaStream_t s) { k_mt_lnorm<<<dim3(1, a.at_n, a.nk), 256, 0, s>>>(a); }
