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
    st->cur_s = a.dvs ? a.dvs[cs] : 0.0;
    st->cur_aa = (av[0] * av[0] + av[1] * av[1] + av[2] * av[2]) / (2.0 * a.c * a.c);
}

// V~ + s dV~ (and its FP32 copy) for steps with a potential change
__global__ void k_vstep(StepArgs a) {
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= a.nvt) return;
    const double s = a.st->cur_s;
    const zd v = zadd(a.vtab[i], zscale(a.dvtab[i], s));
    a.vstep[i] = v;
    if (a.vstep32) a.vstep32[i] = tof(v);
}

// ------------------------------------------------------------ HH(t_k)
__global__ void k_hsub(StepArgs a) {
    const KDev& K = a.kd[blockIdx.z];
    const int n = a.naux;
    const int idx = blockIdx.x * 256 + threadIdx.x;
    if (idx >= n * n) return;
    const int i = idx % n, j = idx / n;
    const DevState* st = a.st;
    const size_t nn = (size_t)n * n;
    zd v = zmk(0.0, 0.0);
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        const double al = st->cur_a[l] / a.c;
        if (al != 0.0) v = zadd(v, zscale(K.psub[l * nn + idx], al));
    }
    if (i == j) v.x += K.eps[i] + st->cur_aa;
    if (a.dv_on) v = zadd(v, K.dvsub[idx]);
    K.hsub[idx] = v;
}

// ------------------------------------------------------------ Chebyshev
// Term n of  sum_n c_n T_n(H~) theta,  H~ = (HH - lam_c)/lam_h:
//   y_1 = H~ y_0, y_n = 2 H~ y_{n-1} - y_{n-2}; acc += c_n y_n.
// One warp per row i; HH is Hermitian so row i is read as column i.
template <int NT>
__global__ void __launch_bounds__(256) k_cheb(StepArgs a, int nt, int last) {
    const KDev& K = a.kd[blockIdx.z];
    const int n = a.naux, ns = a.ns;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + warp;
    if (i >= n) return;
    const size_t vs = (size_t)n * ns;
    const zd* __restrict__ H = K.hsub + (size_t)i * n;
    const zd* yin = (nt == 1) ? K.theta : K.ring + ((nt - 1) % 3) * vs;
    const zd* yp2 = (nt >= 2) ? K.ring + ((nt - 2) % 3) * vs : nullptr;
    zd* yout = K.ring + (nt % 3) * vs;
    const double lc = K.lam[0], lh = K.lam[1];
    const zd cn = K.coef[nt];
    for (int n0 = 0; n0 < ns; n0 += NT) {
        zd acc[NT];
#pragma unroll
        for (int j = 0; j < NT; ++j) acc[j] = zmk(0.0, 0.0);
        for (int jj = lane; jj < n; jj += 32) {
            const zd h = H[jj];
#pragma unroll
            for (int j = 0; j < NT; ++j)
                if (n0 + j < ns) zfmac(acc[j], h, yin[jj + (size_t)(n0 + j) * n]);
        }
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const zd v = warp_zsum(acc[j]);
            const int c = n0 + j;
            if (lane == j && c < ns) {
                const size_t e = i + (size_t)c * n;
                const zd yi = yin[e];
                const zd w = zscale(zsub(v, zscale(yi, lc)), 1.0 / lh);
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
                    const double ph = (a.prop == 0) ? -a.dt * lc : 0.0;
                    K.theta[e] = zmul(zmk(cos(ph), sin(ph)), ac);
                } else {
                    K.acc[e] = ac;
                }
            }
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
// directly into [HC | SC].  Also sum_n f_n Re x_i^* (p_l X)_i for the current.
template <int NT>
__global__ void __launch_bounds__(256) k_local(StepArgs a) {
    const int k = blockIdx.z;
    const KDev& K = a.kd[k];
    const AtomTab& at = *a.at;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * 8 + warp;
    if (row >= at.lrows) return;
    int al = 0;
    while (al + 1 < at.n && at.loff[al + 1] <= row) ++al;
    const int i = row - at.loff[al];
    const int m = at.m[al], na = at.na[al];
    const size_t mm = (size_t)m * m;
    const zd* __restrict__ h = a.h + at.boff[al] + (size_t)i * m;
    const zd* __restrict__ o = a.o + at.boff[al] + (size_t)i * m;
    const zd* __restrict__ p = a.p + 3 * at.boff[al] + (size_t)i * m;
    const zd* __restrict__ dh = a.dh ? a.dh + at.boff[al] + (size_t)i * m : nullptr;
    const DevState* st = a.st;
    const double cx = st->cur_a[0] / a.c, cy = st->cur_a[1] / a.c, cz = st->cur_a[2] / a.c;
    const double aa = st->cur_aa, sdv = st->cur_s;
    const int ns = a.ns, nb = K.nb, ma = at.ma, ng = K.ng;
    const int aoff = at.aoff[al], lo0 = ng + at.looff[al];
    double jc[3] = {0.0, 0.0, 0.0};
    for (int n0 = 0; n0 < ns; n0 += NT) {
        zd aH[NT], aS[NT], aP[3][NT];
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            aH[j] = aS[j] = zmk(0.0, 0.0);
            aP[0][j] = aP[1][j] = aP[2][j] = zmk(0.0, 0.0);
        }
        for (int jj = lane; jj < m; jj += 32) {
            const zd hj = h[jj], oj = o[jj];
            const zd px = p[jj], py = p[mm + jj], pz = p[2 * mm + jj];
            zd he = zadd(hj, zadd(zadd(zscale(px, cx), zscale(py, cy)), zadd(zscale(pz, cz), zscale(oj, aa))));
            if (dh && sdv != 0.0) he = zadd(he, zscale(dh[jj], sdv));
            const zd* xs = (jj < na) ? (K.Q + aoff + jj) : (K.C + lo0 + (jj - na));
            const size_t ld = (jj < na) ? (size_t)ma : (size_t)nb;
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                if (n0 + j >= ns) break;
                const zd x = xs[(size_t)(n0 + j) * ld];
                zfmac(aH[j], he, x);
                zfmac(aS[j], oj, x);
                zfmac(aP[0][j], px, x);
                zfmac(aP[1][j], py, x);
                zfmac(aP[2][j], pz, x);
            }
        }
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const zd zh = warp_zsum(aH[j]);
            const zd zs = warp_zsum(aS[j]);
            const zd q0 = warp_zsum(aP[0][j]);
            const zd q1 = warp_zsum(aP[1][j]);
            const zd q2 = warp_zsum(aP[2][j]);
            const int c = n0 + j;
            if (lane == j && c < ns) {
                zd xi;
                if (i < na) {
                    K.Z[aoff + i + (size_t)c * ma] = zh;
                    K.Z[aoff + i + (size_t)(ns + c) * ma] = zs;
                    xi = K.Q[aoff + i + (size_t)c * ma];
                } else {
                    const int r = lo0 + (i - na);
                    K.Y[r + (size_t)c * nb] = zh;
                    K.Y[r + (size_t)(ns + c) * nb] = zs;
                    xi = K.C[r + (size_t)c * nb];
                }
                const double f = a.occ[c];
                jc[0] += f * (xi.x * q0.x + xi.y * q0.y);
                jc[1] += f * (xi.x * q1.x + xi.y * q1.y);
                jc[2] += f * (xi.x * q2.x + xi.y * q2.y);
            }
        }
    }
    jc[0] = warp_sum(jc[0]);
    jc[1] = warp_sum(jc[1]);
    jc[2] = warp_sum(jc[2]);
    if (lane == 0) {
        double* pj = a.part_jmt + ((size_t)k * at.lrows + row) * 3;
        pj[0] = jc[0];
        pj[1] = jc[1];
        pj[2] = jc[2];
    }
}

// Plane-wave rows, one warp per G:
//   HC_G = |G+k+A/c|^2/2 C_G + sum_G' V~_{G-G'} C_G' + A^H Z_H
//   SC_G = C_G + A^H Z_S
template <typename TA, typename TT, typename TC, int NT>
__global__ void __launch_bounds__(256) k_back(StepArgs a) {
    const int k = blockIdx.z;
    const KDev& K = a.kd[k];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * 8 + warp;
    if (g >= K.ng) return;
    const int ns = a.ns, nb = K.nb, ma = a.ma, ng = K.ng;
    const int* __restrict__ glin = K.glin;
    const int base = glin[g] + a.vt_center;
    const TT* __restrict__ tab;
    const TA* __restrict__ A;
    if constexpr (sizeof(TA) == sizeof(zf)) {
        tab = (const TT*)(a.dv_on ? (const void*)a.vstep32 : (const void*)a.vtab32);
        A = (const TA*)K.amat32 + (size_t)g * ma;
    } else {
        tab = (const TT*)(a.dv_on ? (const void*)a.vstep : (const void*)a.vtab);
        A = (const TA*)K.amat + (size_t)g * ma;
    }
    const zd* __restrict__ X = K.C;
    const zd* __restrict__ Z = K.Z;
    const DevState* st = a.st;
    const double* q = K.gk + 3 * (size_t)g;
    const double dg = 0.5 * (dsq(q[0] + st->cur_a[0] / a.c) + dsq(q[1] + st->cur_a[1] / a.c) +
                             dsq(q[2] + st->cur_a[2] / a.c));
    for (int n0 = 0; n0 < ns; n0 += NT) {
        TC aH[NT], aS[NT];
#pragma unroll
        for (int j = 0; j < NT; ++j) aH[j] = aS[j] = Cx<TC>::zero();
        for (int gp = lane; gp < ng; gp += 32) {
            const TC v = Cx<TC>::from(tab[base - glin[gp]]);
#pragma unroll
            for (int j = 0; j < NT; ++j)
                if (n0 + j < ns) Cx<TC>::fma(aH[j], v, Cx<TC>::from(X[gp + (size_t)(n0 + j) * nb]));
        }
        for (int r = lane; r < ma; r += 32) {
            const TC ar = Cx<TC>::from(A[r]);
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                if (n0 + j >= ns) break;
                Cx<TC>::fmac(aH[j], ar, Cx<TC>::from(Z[r + (size_t)(n0 + j) * ma]));
                Cx<TC>::fmac(aS[j], ar, Cx<TC>::from(Z[r + (size_t)(ns + n0 + j) * ma]));
            }
        }
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            const zd sh = warp_zsum(Cx<TC>::todbl(aH[j]));
            const zd ss = warp_zsum(Cx<TC>::todbl(aS[j]));
            const int c = n0 + j;
            if (lane == j && c < ns) {
                const zd x = X[g + (size_t)c * nb];
                K.Y[g + (size_t)c * nb] = zadd(sh, zscale(x, dg));
                K.Y[g + (size_t)(ns + c) * nb] = zadd(ss, x);
            }
        }
    }
}

// ------------------------------------------------------------ reductions
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

// Per (k, state n, row block): Re c^H (HC), Re c^H (SC), sum_G (G+k)_l |c_G|^2
__global__ void __launch_bounds__(256) k_reduce_full(StepArgs a) {
    __shared__ double sh[32];
    const int k = blockIdx.z, n = blockIdx.y, b = blockIdx.x;
    const KDev& K = a.kd[k];
    const int nb = K.nb, ng = K.ng, ns = a.ns;
    const int per = (nb + RB_FULL - 1) / RB_FULL;
    const int r0 = b * per, r1 = min(nb, r0 + per);
    double e = 0.0, s = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const zd c = K.C[r + (size_t)n * nb];
        const zd hc = K.Y[r + (size_t)n * nb];
        const zd sc = K.Y[r + (size_t)(ns + n) * nb];
        e += c.x * hc.x + c.y * hc.y;
        s += c.x * sc.x + c.y * sc.y;
        if (r < ng) {
            const double w = c.x * c.x + c.y * c.y;
            const double* q = K.gk + 3 * (size_t)r;
            jx += q[0] * w;
            jy += q[1] * w;
            jz += q[2] * w;
        }
    }
    e = block_sum(e, sh);
    s = block_sum(s, sh);
    jx = block_sum(jx, sh);
    jy = block_sum(jy, sh);
    jz = block_sum(jz, sh);
    if (threadIdx.x == 0) {
        double* pf = a.part_full + (((size_t)k * ns + n) * RB_FULL + b) * 5;
        pf[0] = e;
        pf[1] = s;
        pf[2] = jx;
        pf[3] = jy;
        pf[4] = jz;
    }
}

// max |theta^H theta~ - I| (= max |C^H S C - I| for C = CC theta) and
// max |theta~ - theta| per k-point
__global__ void __launch_bounds__(256) k_normred(StepArgs a) {
    __shared__ double sh[32];
    const int k = blockIdx.x;
    const KDev& K = a.kd[k];
    const int ns = a.ns, n = a.naux;
    double d1 = 0.0, d2 = 0.0;
    for (int e = threadIdx.x; e < ns * ns; e += blockDim.x) {
        zd g = K.gram[e];
        if (e % ns == e / ns) g.x -= 1.0;
        d1 = fmax(d1, hypot(g.x, g.y));
    }
    for (int e = threadIdx.x; e < n * ns; e += blockDim.x) {
        const zd d = zsub(K.theta_t[e], K.theta[e]);
        d2 = fmax(d2, hypot(d.x, d.y));
    }
    d1 = block_max(d1, sh);
    d2 = block_max(d2, sh);
    if (threadIdx.x == 0) {
        a.part_norm[2 * k] = d1;
        a.part_norm[2 * k + 1] = d2;
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

// J contributions from the subspace: sum_n f_n Re theta_in^* ((PP_l + A_l/c) theta)_in,
// one warp per (l, i)
__global__ void __launch_bounds__(256) k_subj(StepArgs a) {
    const int k = blockIdx.z;
    const KDev& K = a.kd[k];
    const int n = a.naux, ns = a.ns;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * 8 + warp;
    if (row >= 3 * n) return;
    const int l = row / n, i = row % n;
    const zd* __restrict__ P = K.psub + (size_t)l * n * n + (size_t)i * n;
    const double al = a.st->cur_a[l] / a.c;
    double tot = 0.0;
    for (int c = 0; c < ns; ++c) {
        zd v = zmk(0.0, 0.0);
        const zd* th = K.theta + (size_t)c * n;
        for (int j = lane; j < n; j += 32) zfmac(v, P[j], th[j]);
        v = warp_zsum(v);
        const zd ti = th[i];
        tot += a.occ[c] * (ti.x * (v.x + al * ti.x) + ti.y * (v.y + al * ti.y));
    }
    if (lane == 0) a.part_sub[((size_t)k * 3 + l) * n + i] = tot;
}

// Sum the step's partials over k-points (weights w_k), update the dipole by
// the trapezoid rule (Eq. dipole) and append the record.  One block.
__global__ void __launch_bounds__(256) k_finalize(StepArgs a, int set_gs) {
    __shared__ double sh[32];
    DevState* st = a.st;
    const int ns = a.ns, n = a.naux, lrows = a.lrows;
    double J[3] = {0, 0, 0}, JF[3] = {0, 0, 0}, E = 0.0, ndev = 0.0, res = 0.0, dtcr = 1e300;
    const double io = -1.0 / a.omega;
    for (int k = 0; k < a.nk; ++k) {
        const KDev& K = a.kd[k];
        const double w = a.wk[k];
        double js[3];
        for (int l = 0; l < 3; ++l) {
            double v = 0.0;
            for (int i = threadIdx.x; i < n; i += blockDim.x) v += a.part_sub[((size_t)k * 3 + l) * n + i];
            js[l] = block_sum(v, sh);
            J[l] += w * io * js[l];
        }
        if (set_gs) continue;
        double e = 0.0, sf = 0.0, ji[3] = {0, 0, 0};
        for (int idx = threadIdx.x; idx < ns * RB_FULL; idx += blockDim.x) {
            const int c = idx / RB_FULL;
            const double f = a.occ[c];
            const double* pf = a.part_full + ((size_t)k * ns * RB_FULL + idx) * 5;
            e += f * pf[0];
            sf += f * pf[1];
            ji[0] += f * pf[2];
            ji[1] += f * pf[3];
            ji[2] += f * pf[4];
        }
        e = block_sum(e, sh);
        sf = block_sum(sf, sh);
        double jm[3];
        for (int l = 0; l < 3; ++l) {
            double v = 0.0;
            for (int r = threadIdx.x; r < lrows; r += blockDim.x) v += a.part_jmt[((size_t)k * lrows + r) * 3 + l];
            jm[l] = block_sum(v, sh);
            const double jil = block_sum(ji[l], sh);
            JF[l] += w * io * (jil + jm[l] + st->cur_a[l] / a.c * sf);
        }
        E += w * e;
        ndev = fmax(ndev, a.part_norm[2 * k]);
        res = fmax(res, a.part_norm[2 * k + 1]);
        double dk;
        if (a.prop == 1) {
            dk = 0.2 / (K.eval[n - 1] - K.eval[0]);
        } else {
            dk = 0.2 / (2.0 * K.lam[1]);
        }
        dtcr = fmin(dtcr, dk);
    }
    if (threadIdx.x != 0) return;
    if (set_gs) {
        for (int l = 0; l < 3; ++l) st->j_gs[l] = J[l];
        return;
    }
    const double t = st->t + a.dt;
    double* r = a.rec + (size_t)st->rec_count * RTD_REC_STRIDE;
    r[REC_T] = t;
    for (int l = 0; l < 3; ++l) {
        const double jind = J[l] - st->j_gs[l];
        st->dmu[l] += a.omega * a.dt * 0.5 * (st->jind_prev[l] + jind);
        st->jind_prev[l] = jind;
        r[REC_J + l] = J[l];
        r[REC_JF + l] = JF[l];
        r[REC_DMU + l] = st->dmu[l];
    }
    r[REC_E] = E;
    r[REC_NDEV] = ndev;
    r[REC_RES] = res;
    r[REC_DTCR] = dtcr;
    st->t = t;
    st->rec_count += 1;
    st->gstep += 1;
    st->cstep += 1;
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
void launch_set_cur(const StepArgs& a, cudaStream_t s) { k_set_cur<<<1, 1, 0, s>>>(a); }

void launch_prep_coef(const StepArgs& a, cudaStream_t s) {
    if (a.prop == 1) return;
    k_coef<<<a.nk, 32, 0, s>>>(a);
}

void launch_subspace_current(const StepArgs& a, int set_gs, cudaStream_t s) {
    dim3 g((3 * a.naux + 7) / 8, 1, a.nk);
    k_subj<<<g, 256, 0, s>>>(a);
    k_finalize<<<1, 256, 0, s>>>(a, set_gs);
}

static inline void mark(TraceHook* tr, const char* name, cudaStream_t s) {
    if (!tr || tr->n >= tr->cap) return;
    tr->names[tr->n] = name;
    cudaEventRecord(tr->ev[tr->n], s);
    tr->n += 1;
}

void launch_operator_pass(const StepArgs& a, const StepPlan& p, cudaStream_t s, TraceHook* tr) {
    const bool f32 = a.prec == 1;
    // Q = A C_G (matching coefficients applied to the plane-wave rows)
    launch_gemm_nn(p.gd_fwd, a.nk, a.ma, p.maxng, a.ns, p.kc_fwd, p.part, 0, f32, nullptr, s);
    mark(tr, "gemm_forward", s);
    launch_split_reduce(p.gd_fwd, a.nk, a.ma, a.ns, p.kc_fwd, p.part, 0, s);
    mark(tr, "split_reduce_forward", s);
    if (a.lrows > 0) {
        dim3 g((a.lrows + 7) / 8, 1, a.nk);
        if (a.ns <= 2) k_local<2><<<g, 256, 0, s>>>(a);
        else k_local<4><<<g, 256, 0, s>>>(a);
        mark(tr, "local_mt", s);
    }
    {
        dim3 g((p.maxng + 7) / 8, 1, a.nk);
        if (f32) {
            if (a.ns <= 2) k_back<zf, zf, zf, 2><<<g, 256, 0, s>>>(a);
            else if (a.ns <= 4) k_back<zf, zf, zf, 4><<<g, 256, 0, s>>>(a);
            else k_back<zf, zf, zf, 8><<<g, 256, 0, s>>>(a);
        } else {
            if (a.ns <= 2) k_back<zd, zd, zd, 2><<<g, 256, 0, s>>>(a);
            else if (a.ns <= 4) k_back<zd, zd, zd, 4><<<g, 256, 0, s>>>(a);
            else k_back<zd, zd, zd, 8><<<g, 256, 0, s>>>(a);
        }
        mark(tr, "back_toeplitz", s);
    }
}

void launch_step(const StepArgs& a, const StepPlan& p, cudaStream_t s, int* nlaunch, TraceHook* tr) {
    int nl = 0;
    const bool f32 = a.prec == 1;
    const int nn = a.naux * a.naux;
    k_set_cur<<<1, 1, 0, s>>>(a);
    mark(tr, "set_cur", s);
    ++nl;
    if (a.dv_on) {
        // Eq. v_MT and Eq. v_interstitial rebuilt from the scaled blocks:
        // dVV = L^H (s dh) L + CC_G^H (s dV~ * CC_G)
        k_vstep<<<(a.nvt + 255) / 256, 256, 0, s>>>(a);
        mark(tr, "dv_table", s);
        launch_gemm_nn(p.gd_dvw, p.n_dvw, p.maxm, p.maxm, a.naux, 0, nullptr, 0, false,
                       &a.st->cur_s, s);
        mark(tr, "dv_mt_blocks", s);
        launch_gemm_cn(p.gd_dvg, a.nk, a.naux, a.lrows, a.naux, 0, nullptr, 0, false, nullptr, s);
        mark(tr, "dv_mt_project", s);
        launch_toeplitz(a.kd, p.td_dv, a.nk, p.maxng, a.naux, a.dvtab, a.vt_center, 0, 0,
                        &a.st->cur_s, s);
        mark(tr, "dv_interstitial_toeplitz", s);
        launch_gemm_cn(p.gd_dvi, a.nk, a.naux, p.maxng, a.naux, 0, nullptr, 1, false, nullptr, s);
        mark(tr, "dv_interstitial_project", s);
        nl += 5;
    }
    k_hsub<<<dim3((nn + 255) / 256, 1, a.nk), 256, 0, s>>>(a);
    mark(tr, "hsub", s);
    ++nl;
    if (a.prop == 1) {
        launch_jacobi(p.jac_mats, p.jac_vals, p.jac_vecs, a.nk, a.naux, p.max_sweeps, p.d_flag, s);
        mark(tr, "jacobi", s);
        launch_gemm_cn(p.gd_evh, a.nk, a.naux, a.naux, a.ns, 0, nullptr, 0, false, nullptr, s);
        k_eigphase<<<dim3((a.naux * a.ns + 255) / 256, 1, a.nk), 256, 0, s>>>(a);
        launch_gemm_nn(p.gd_evn, a.nk, a.naux, a.naux, a.ns, 0, nullptr, 0, false, nullptr, s);
        mark(tr, "eig_apply", s);
        nl += 4;
    } else {
        dim3 g((a.naux + 7) / 8, 1, a.nk);
        for (int t = 1; t < a.nterms; ++t) {
            const int last = (t == a.nterms - 1);
            if (a.ns <= 2) k_cheb<2><<<g, 256, 0, s>>>(a, t, last);
            else if (a.ns <= 4) k_cheb<4><<<g, 256, 0, s>>>(a, t, last);
            else k_cheb<8><<<g, 256, 0, s>>>(a, t, last);
            mark(tr, "chebyshev_term", s);
            ++nl;
        }
    }
    // C = CC theta (Eq. approximation_coefficients)
    launch_gemm_nn(p.gd_expand, a.nk, p.maxnb, a.naux, a.ns, 0, nullptr, 0, f32, nullptr, s);
    mark(tr, "gemm_expand", s);
    ++nl;
    launch_operator_pass(a, p, s, tr);
    nl += 4;
    k_reduce_full<<<dim3(RB_FULL, a.ns, a.nk), 256, 0, s>>>(a);
    mark(tr, "reduce_full", s);
    ++nl;
    // theta~ = CC^H (S C)
    launch_gemm_cn(p.gd_proj, a.nk, a.naux, p.maxnb, a.ns, p.kc_proj, p.part, 0, f32, nullptr, s);
    mark(tr, "gemm_project", s);
    launch_split_reduce(p.gd_proj, a.nk, a.naux, a.ns, p.kc_proj, p.part, 0, s);
    mark(tr, "split_reduce_project", s);
    launch_gemm_cn(p.gd_g1, a.nk, a.ns, a.naux, a.ns, 0, nullptr, 0, false, nullptr, s);
    mark(tr, "gram", s);
    k_normred<<<a.nk, 256, 0, s>>>(a);
    mark(tr, "norm_residual", s);
    nl += 4;
    if (a.reproject) {
        launch_gemm_cn(p.gd_g2, a.nk, a.ns, a.naux, a.ns, 0, nullptr, 0, false, nullptr, s);
        k_reproj<<<dim3((a.naux * a.ns + 255) / 256, 1, a.nk), 256, 0, s>>>(a);
        mark(tr, "reproject", s);
        nl += 2;
    }
    {
        dim3 g((3 * a.naux + 7) / 8, 1, a.nk);
        k_subj<<<g, 256, 0, s>>>(a);
        mark(tr, "subspace_current", s);
        k_finalize<<<1, 256, 0, s>>>(a, 0);
        mark(tr, "finalize", s);
    }
    nl += 2;
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
