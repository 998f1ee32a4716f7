// Reverse mode through the subspace step, for d(gdir . dmu(T)) / dA_k.
//
// The forward map of one step is theta' = beta sum_n c_n y_n with
// y_0 = theta, y_1 = H~ y_0, y_n = 2 H~ y_{n-1} - y_{n-2}, H~ = (HH - lc)/lh,
// beta = e^{-i dt lc} (the Chebyshev series of exp(-i HH dt), same
// coefficients as the step).  Its exact adjoint for an output gradient o
// (convention dL = Re <o, d theta'>) is the reversed recurrence
//   ybar_n = conj(beta c_n) o,  for n = N-1 .. 2:  ybar_{n-1} += 2 H~ ybar_n,
//   ybar_{n-2} -= ybar_n;  ybar_0 += H~ ybar_1;  theta-bar = ybar_0,
// and the matrix gradient Gbar = sum_n f_n ybar_n y_{n-1}^H (f_1 = 1, f_n = 2),
// with dL/dA_l = Re tr(Gbar^H dH~/dA_l), dH~/dA_l = (PP_l / c + A_l/c^2 I) / lh.
#include "rtd.h"

// y_nt = H~ y_0 (nt = 1) or 2 H~ y_{nt-1} - y_{nt-2}; one block per row (k, i).
__global__ void __launch_bounds__(128) k_adj_fwd_term(StepArgs a, zd* __restrict__ Yh, int nterm, int nt) {
    __shared__ double red[4][2];
    const int k = blockIdx.z, i = blockIdx.x;
    const KDev& K = a.kd[k];
    const int n = a.naux, ns = a.ns;
    const size_t vs = (size_t)n * ns;
    zd* Y = Yh + (size_t)k * nterm * vs;
    const zd* H = K.hsub + (size_t)i * n;
    const double lc = K.lam[0], ilh = K.lam[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int c = 0; c < ns; ++c) {
        const zd* yin = Y + (size_t)(nt - 1) * vs + (size_t)c * n;
        zd v = zmk(0.0, 0.0);
        for (int j = tid; j < n; j += 128) zfmac(v, H[j], yin[j]);
        v = warp_zsum(v);
        if (lane == 0) {
            red[warp][0] = v.x;
            red[warp][1] = v.y;
        }
        __syncthreads();
        if (tid == 0) {
            const zd s = zmk(red[0][0] + red[1][0] + red[2][0] + red[3][0], red[0][1] + red[1][1] + red[2][1] + red[3][1]);
            const zd w = zscale(zsub(s, zscale(yin[i], lc)), ilh);
            zd y = w;
            if (nt >= 2) y = zsub(zscale(w, 2.0), Y[(size_t)(nt - 2) * vs + (size_t)c * n + i]);
            Y[(size_t)nt * vs + (size_t)c * n + i] = y;
        }
        __syncthreads();
    }
}

// ybar_n = conj(beta c_n) o for every n
__global__ void k_adj_bwd_init(StepArgs a, zd* __restrict__ Yb, const zd* __restrict__ lam, int nterm) {
    const int k = blockIdx.z;
    const KDev& K = a.kd[k];
    const size_t vs = (size_t)a.naux * a.ns;
    const int e = blockIdx.x * 256 + threadIdx.x;
    if (e >= (int)vs) return;
    const zd beta = (a.prop == 0) ? zmk(K.lam[3], K.lam[4]) : zmk(1.0, 0.0);
    const zd o = lam[(size_t)k * vs + e];
    for (int t = 0; t < nterm; ++t) {
        const zd bc = zconj(zmul(beta, K.coef[t]));
        Yb[((size_t)k * nterm + t) * vs + e] = zmul(bc, o);
    }
}

// reverse of term nt: ybar_{nt-1} += f H~ ybar_nt (f = 2, or 1 for nt = 1),
// ybar_{nt-2} -= ybar_nt; one block per row (k, i).
__global__ void __launch_bounds__(128) k_adj_bwd_term(StepArgs a, zd* __restrict__ Yb, int nterm, int nt) {
    __shared__ double red[4][2];
    const int k = blockIdx.z, i = blockIdx.x;
    const KDev& K = a.kd[k];
    const int n = a.naux, ns = a.ns;
    const size_t vs = (size_t)n * ns;
    zd* Y = Yb + (size_t)k * nterm * vs;
    const zd* H = K.hsub + (size_t)i * n;
    const double lc = K.lam[0], ilh = K.lam[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int c = 0; c < ns; ++c) {
        const zd* yb = Y + (size_t)nt * vs + (size_t)c * n;
        zd v = zmk(0.0, 0.0);
        for (int j = tid; j < n; j += 128) zfmac(v, H[j], yb[j]);
        v = warp_zsum(v);
        if (lane == 0) {
            red[warp][0] = v.x;
            red[warp][1] = v.y;
        }
        __syncthreads();
        if (tid == 0) {
            const zd s = zmk(red[0][0] + red[1][0] + red[2][0] + red[3][0], red[0][1] + red[1][1] + red[2][1] + red[3][1]);
            const zd w = zscale(zsub(s, zscale(yb[i], lc)), ilh);
            const double f = (nt >= 2) ? 2.0 : 1.0;
            zd* p1 = Y + (size_t)(nt - 1) * vs + (size_t)c * n + i;
            *p1 = zadd(*p1, zscale(w, f));
            if (nt >= 2) {
                zd* p2 = Y + (size_t)(nt - 2) * vs + (size_t)c * n + i;
                *p2 = zsub(*p2, yb[i]);
            }
        }
        __syncthreads();
    }
}

// Per element (i, j) of HH: G_ij = sum_n f_n sum_s ybar_n[i,s] conj(y_{n-1}[j,s]);
// the block sums Re conj(G_ij) PP_l[i,j] (l = x,y,z) and Re G_ii into
// part[(k * gridDim.x + block) * 4 + {0,1,2,3}].
__global__ void __launch_bounds__(256) k_adj_grad(StepArgs a, const zd* __restrict__ Yh, const zd* __restrict__ Yb,
                                                  int nterm, double* __restrict__ part) {
    __shared__ double sh[8][4];
    const int k = blockIdx.z;
    const KDev& K = a.kd[k];
    const int n = a.naux, ns = a.ns;
    const size_t vs = (size_t)n * ns, nn = (size_t)n * n;
    const zd* Y = Yh + (size_t)k * nterm * vs;
    const zd* B = Yb + (size_t)k * nterm * vs;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (size_t e = (size_t)blockIdx.x * 256 + threadIdx.x; e < nn; e += (size_t)gridDim.x * 256) {
        const int i = (int)(e % n), j = (int)(e / n);
        zd g = zmk(0.0, 0.0);
        for (int t = 1; t < nterm; ++t) {
            const double f = (t >= 2) ? 2.0 : 1.0;
            zd gt = zmk(0.0, 0.0);
            for (int c = 0; c < ns; ++c)
                zfma(gt, B[(size_t)t * vs + (size_t)c * n + i], zconj(Y[(size_t)(t - 1) * vs + (size_t)c * n + j]));
            g = zadd(g, zscale(gt, f));
        }
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const zd p = K.psub[l * nn + e];
            acc[l] += g.x * p.x + g.y * p.y;
        }
        if (i == j) acc[3] += g.x;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const double v = warp_sum(acc[q]);
        if (lane == 0) sh[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += sh[w][threadIdx.x];
        part[((size_t)k * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = v;
    }
}

// Adjoint source of the current at t_m: for every k, row i and state s
//   lam[i,s] += cfac * w_k f_s ((sum_l g_l PP_l) theta + sm theta)[i,s]
// and per row the weighted norm w_k sum_s f_s |theta[i,s]|^2 into nrm.
// One warp per row.
__global__ void __launch_bounds__(256) k_adj_jterm(StepArgs a, zd* __restrict__ lam, const zd* __restrict__ theta,
                                                   double g0, double g1, double g2, double sm, double cfac,
                                                   double* __restrict__ nrm) {
    const int k = blockIdx.z;
    const KDev& K = a.kd[k];
    const int n = a.naux, ns = a.ns;
    const size_t vs = (size_t)n * ns, nn = (size_t)n * n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + warp;
    if (i >= n) return;
    const zd* th = theta + (size_t)k * vs;
    zd* lm = lam + (size_t)k * vs;
    const double wk = a.wk[k];
    double nr = 0.0;
    for (int c = 0; c < ns; ++c) {
        zd v = zmk(0.0, 0.0);
        for (int j = lane; j < n; j += 32) {
            const size_t off = (size_t)i * n + j;  // column i of the Hermitian PP_l
            const zd p = zadd(zadd(zscale(K.psub[off], g0), zscale(K.psub[nn + off], g1)), zscale(K.psub[2 * nn + off], g2));
            zfmac(v, p, th[(size_t)c * n + j]);
        }
        v = warp_zsum(v);
        if (lane == 0) {
            const zd ti = th[(size_t)c * n + i];
            const double f = wk * a.occ[c];
            const zd src = zadd(v, zscale(ti, sm));
            lm[(size_t)c * n + i] = zadd(lm[(size_t)c * n + i], zscale(src, cfac * f));
            nr += f * (ti.x * ti.x + ti.y * ti.y);
        }
    }
    if (lane == 0) nrm[(size_t)k * n + i] = nr;
}

void launch_adj_fwd_term(const StepArgs& a, zd* Yh, int nterm, int nt, cudaStream_t s) {
    k_adj_fwd_term<<<dim3(a.naux, 1, a.nk), 128, 0, s>>>(a, Yh, nterm, nt);
}
void launch_adj_bwd_init(const StepArgs& a, zd* Yb, const zd* lam, int nterm, cudaStream_t s) {
    k_adj_bwd_init<<<dim3((a.naux * a.ns + 255) / 256, 1, a.nk), 256, 0, s>>>(a, Yb, lam, nterm);
}
void launch_adj_bwd_term(const StepArgs& a, zd* Yb, int nterm, int nt, cudaStream_t s) {
    k_adj_bwd_term<<<dim3(a.naux, 1, a.nk), 128, 0, s>>>(a, Yb, nterm, nt);
}
void launch_adj_grad(const StepArgs& a, const zd* Yh, const zd* Yb, int nterm, double* part, int nblk,
                     cudaStream_t s) {
    k_adj_grad<<<dim3(nblk, 1, a.nk), 256, 0, s>>>(a, Yh, Yb, nterm, part);
}
void launch_adj_jterm(const StepArgs& a, zd* lam, const zd* theta, const double* g, double sm, double cfac,
                      double* nrm, cudaStream_t s) {
    k_adj_jterm<<<dim3((a.naux + 7) / 8, 1, a.nk), 256, 0, s>>>(a, lam, theta, g[0], g[1], g[2], sm, cfac, nrm);
}
