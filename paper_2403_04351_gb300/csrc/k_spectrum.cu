// Post-processing of the recorded current: the dynamical polarizability of
// Eq. polarizability, alpha_{l l'}(w) = (i Omega / w) J_l(w) / E_l'(w), with
// the time series taken to the frequency domain by the damped discrete
// transform F(w) = dt sum_n f(t_n) e^{(i w - eta) t_n}.
#include "rtd.h"
#include "rttddft.h"

#include <string>
#include <vector>

#define SPEC_THREADS 256

// one block per frequency: the six transforms (J_x,y,z and E_x,y,z) summed
// over the samples in a fixed order, then alpha
__global__ void __launch_bounds__(SPEC_THREADS) k_spectrum(int nt, double t0, double dt, const double* __restrict__ j,
                                                         const double* __restrict__ e, double eta,
                                                         const double* __restrict__ w, double cell, zd* out_j,
                                                         zd* out_e, zd* alpha) {
    __shared__ double red[SPEC_THREADS / 32][16];
    __shared__ zd ft[6];
    const int iw = blockIdx.x;
    const double om = w[iw];
    double v[16];  // 12 sums, padded to the power of two the warp reduction takes
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = 0.0;
    for (int n = threadIdx.x; n < nt; n += SPEC_THREADS) {
        const double t = t0 + n * dt;
        double sn, cs;
        sincos(om * t, &sn, &cs);
        const double damp = exp(-eta * t);
        const double fr = damp * cs, fi = damp * sn;
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const double jl = j[3 * (size_t)n + l], el = e[3 * (size_t)n + l];
            v[2 * l] += jl * fr;
            v[2 * l + 1] += jl * fi;
            v[6 + 2 * l] += el * fr;
            v[6 + 2 * l + 1] += el * fi;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_sum_store<double, 16>(v, lane, red[warp]);
    __syncthreads();
    if (threadIdx.x < 6) {
        double re = 0.0, im = 0.0;
        for (int q = 0; q < SPEC_THREADS / 32; ++q) {
            re += red[q][2 * threadIdx.x];
            im += red[q][2 * threadIdx.x + 1];
        }
        ft[threadIdx.x] = zmk(re * dt, im * dt);
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        if (out_j) out_j[3 * (size_t)iw + threadIdx.x] = ft[threadIdx.x];
        if (out_e) out_e[3 * (size_t)iw + threadIdx.x] = ft[3 + threadIdx.x];
    }
    if (alpha && threadIdx.x < 9) {
        const int l = threadIdx.x / 3, lp = threadIdx.x % 3;
        const zd jl = ft[l], el = ft[3 + lp];
        const double d = el.x * el.x + el.y * el.y;
        zd a = zmk(0.0, 0.0);
        if (d > 0.0) {
            // (i Omega / w) * jl / el = (i Omega / w) * jl * conj(el) / |el|^2
            const zd q = zmk((jl.x * el.x + jl.y * el.y) / d, (jl.y * el.x - jl.x * el.y) / d);
            const double f = cell / om;
            a = zmk(-f * q.y, f * q.x);
        }
        alpha[9 * (size_t)iw + threadIdx.x] = a;
    }
}

static bool on_device(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

extern "C" int rttddft_polarizability(int n_t, double t0, double dt, const double* j_ind, const double* e_field,
                                      double eta, int n_w, const double* w, double omega_cell, double* out_j,
                                      double* out_e, double* alpha, void* cuda_stream) {
    if (n_t < 1 || n_w < 1 || !(dt > 0.0) || !(omega_cell > 0.0) || !(eta >= 0.0) || !j_ind || !e_field || !w)
        return RTTDDFT_ERR_ARG;
    if (!on_device(w)) {
        for (int i = 0; i < n_w; ++i)
            if (!(w[i] > 0.0)) return RTTDDFT_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    std::vector<void*> tmp;
    auto release = [&]() {
        for (void* p : tmp) cudaFree(p);
    };
    // inputs: device pointers are read in place, host arrays staged
    auto stage_in = [&](const double* h, size_t n, const double** d) -> bool {
        if (on_device(h)) {
            *d = h;
            return true;
        }
        void* p = nullptr;
        if (cudaMalloc(&p, n * sizeof(double)) != cudaSuccess) return false;
        tmp.push_back(p);
        if (cudaMemcpyAsync(p, h, n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) return false;
        *d = (const double*)p;
        return true;
    };
    auto stage_out = [&](double* h, size_t n, zd** d) -> bool {
        if (!h) {
            *d = nullptr;
            return true;
        }
        if (on_device(h)) {
            *d = (zd*)h;
            return true;
        }
        void* p = nullptr;
        if (cudaMalloc(&p, n * sizeof(double)) != cudaSuccess) return false;
        tmp.push_back(p);
        *d = (zd*)p;
        return true;
    };
    const double *dj = nullptr, *de = nullptr, *dw = nullptr;
    zd *oj = nullptr, *oe = nullptr, *oa = nullptr;
    if (!stage_in(j_ind, 3 * (size_t)n_t, &dj) || !stage_in(e_field, 3 * (size_t)n_t, &de) ||
        !stage_in(w, (size_t)n_w, &dw) || !stage_out(out_j, 6 * (size_t)n_w, &oj) ||
        !stage_out(out_e, 6 * (size_t)n_w, &oe) || !stage_out(alpha, 18 * (size_t)n_w, &oa)) {
        cudaStreamSynchronize(st);
        release();
        return RTTDDFT_ERR_CUDA;
    }
    k_spectrum<<<n_w, SPEC_THREADS, 0, st>>>(n_t, t0, dt, dj, de, eta, dw, omega_cell, oj, oe, oa);
    bool ok = cudaGetLastError() == cudaSuccess;
    auto back = [&](double* h, zd* d, size_t n) {
        if (h && (void*)d != (void*)h)
            ok = ok && cudaMemcpyAsync(h, d, n * sizeof(double), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    };
    back(out_j, oj, 6 * (size_t)n_w);
    back(out_e, oe, 6 * (size_t)n_w);
    back(alpha, oa, 18 * (size_t)n_w);
    ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
    release();
    return ok ? RTTDDFT_OK : RTTDDFT_ERR_CUDA;
}
