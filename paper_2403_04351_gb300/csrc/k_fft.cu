// Interstitial convolution of Eq. v_interstitial by fast Fourier transforms:
// the route that the paper recommends for large plane-wave cut-offs (Sec. 3,
// the cost of the interstitial term, and the FFT against matrix-product
// comparison).
//
//   Y_G = sum_G' V~_{G-G'} C_G'     for G in the plane-wave set of a k-point
//
// The G - G' differences of one k-point lie in the table box |d_i| <= e_i,
// so on a periodic grid of F_i >= 2 e_i + 1 points per axis every difference
// has its own residue (d_i mod F_i).  With V~ placed on the grid by residue,
// v(r_j) = F^-3 sum_d V~_d e^{+2 pi i d.j/F} (set-up), the circular
// convolution equals the sum above:
//   c(r_j) = sum_G' C_G' e^{+2 pi i G'.j/F}                (inverse transform)
//   Y_G    = sum_j e^{-2 pi i G.j/F} v(r_j) c(r_j)          (forward transform)
// Both transforms are pruned to the G set: C is non-zero on the lines
// (n1, n2) and planes n1 that hold a G vector, and Y is needed only there.
// Five passes per product, each a batch of 1-D transforms in shared memory
// (Stockham autosort, radices 2, 3, 4, 5):
//   A  inverse along axis 3, lines holding a G        (scatter C_G)
//   B  inverse along axis 2, planes holding a G
//   C  along axis 1 on every (r2, r3): inverse, times v(r), forward
//   D  forward along axis 2, kept on the lines holding a G
//   E  forward along axis 3                           (gather Y_G)
// All k-points and columns of a product run in the same five launches.
#include "rtd.h"
#include "rttddft.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <string>
#include <vector>

#define FFT_LPB 16        // lines per block at most
#define FFT_BLK_PTS 2048  // points of a line block at most: lines per block = min(16, 2048 / L)
#define FFT_THREADS 128
#define FFT_PV (FFT_BLK_PTS / FFT_THREADS)  // points of a block per thread
#define FFT_PTHREADS 256  // plane kernels
#define FFT_MAX_N 512     // longest axis
#define FFT_MAX_ST 8

// lines of length L per block of a line pass
static inline int fft_lpb(int L) { return std::min(FFT_LPB, FFT_BLK_PTS / std::max(L, 1)); }

struct FftK {
    int nline, nplane;
    const int* lg0;       // [nline + 1] first entry of each line in line order
    const int* gperm;     // [ng] G index of each entry in line order
    const int* lpos;      // [ng] line * F3 + residue of n3, per entry
    const int* plane_of;  // [F1] plane of a residue of n1, or -1
    const int* line_of;   // [nplane][F2] line of (plane, residue of n2), or -1
    const int* pl0;       // [nplane + 1] first line of each plane
    const int* lr2;       // [nline] residue of n2 of each line
};

struct FftArgs {
    int F1, F2, F3;
    int nst[3];
    int rad[3][FFT_MAX_ST];
    int lpb[3];             // lines per block of the passes along each axis
    const void* w[3];       // twiddles e^{-2 pi i m / F_a}, m < F_a (FP64 or FP32 complex)
    const FftK* fk;         // per k-point of the launch
    const ToepDesc* td;     // per k-point: source X (ld ldx) and destination Y (ld ldy)
    void* b3;               // [k][col][max_lines][F3]
    void* b2;               // [k][col][max_planes][F2][F3]
    size_t b3_col, b2_col;  // elements per column
    int ncol;
    int vmode;              // 0: v (+ s vd when use_vd), 1: s vd alone
    int use_vd;
    const void* v;          // potential on the grid (complex, FP64 or FP32)
    const void* vd;
    const double* s;        // scale of vd (device)
};

struct FftPlan {
    int F[3];
    int nst[3];
    int rad[3][FFT_MAX_ST];
    int prec;  // 0 FP64, 1 FP32
    int nk;
    int max_lines, max_planes;
    int ncol;
    int fused = 0;  // 1: axes 3 and 2 of a plane in one launch (three launches per product)
    float ms_split = 0.f, ms_fused = 0.f;  // set-up timings of both launch sets
    zd* w64[3] = {nullptr, nullptr, nullptr};
    zf* w32[3] = {nullptr, nullptr, nullptr};
    zd* v64 = nullptr;
    zf* v32 = nullptr;
    zd* vd64 = nullptr;
    zf* vd32 = nullptr;
    FftK* d_fk = nullptr;
    void* b3 = nullptr;
    void* b2 = nullptr;
    std::vector<void*> tables;  // per-k index arrays
    // Hartree feedback: density grid (forward transformed), its value at the
    // start, the box extents, the reciprocal vectors, the l1 accumulator
    // (the density and its potential are FP64 in every form: the change n(t) - n(0)
    // is a small difference of two densities, which FP32 rounding would swamp)
    zd* rho = nullptr;
    zd* rho0 = nullptr;
    zd* b3d = nullptr;  // FP64 transform buffers of the density (FP32 plans only)
    zd* b2d = nullptr;
    int fused_d = 0;    // the density's plane pass fused (FP64 plane in shared memory)
    double* l1 = nullptr;
    int hartree = 0;
    int e[3] = {0, 0, 0};
    double recip[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    double omega = 1.0, bound = 0.0;
};

// ---------------------------------------------------------------- complex ops
template <typename C> struct Rt;
template <> struct Rt<zd> { typedef double R; };
template <> struct Rt<zf> { typedef float R; };
template <typename C> __device__ __forceinline__ C cmk(typename Rt<C>::R x, typename Rt<C>::R y) {
    C r;
    r.x = x;
    r.y = y;
    return r;
}
template <typename C> __device__ __forceinline__ C cad(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csb(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cml(C a, C b) {
    return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// i * z * sgn
template <typename C> __device__ __forceinline__ C cis(C z, typename Rt<C>::R sg) { return cmk<C>(-sg * z.y, sg * z.x); }
template <typename C> __device__ __forceinline__ C cwt(const C* W, int i, bool inv) {
    C w = W[i];
    if (inv) w.y = -w.y;
    return w;
}
__device__ __forceinline__ zd cvt(zd a, zd) { return a; }
__device__ __forceinline__ zf cvt(zd a, zf) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ zd todz(zd a) { return a; }
__device__ __forceinline__ zd todz(zf a) { return zmk(a.x, a.y); }

// Stockham autosort, decimation in frequency: nl lines of length L stored
// line by line in x (y is scratch of the same size).  A stage of radix R on
// sub-transforms of length n = L/s (s interleaved sequences) maps
//   x[q + s(p + r m)]  ->  y[q + s(R p + t)] = w_n^{p t} sum_r x[q + s(p + r m)] w_R^{r t},
// m = n/R, p < m, q < s; after the last stage the transform is in natural
// order.  inv selects e^{+}.  Element j of line l sits at l ls + j es (in x and
// y alike).  Returns the buffer holding the result.
template <typename C>
__device__ C* fft_lines_s(C* x, C* y, int nl, int L, int ls, int es, const int* rad, int nst, const C* W,
                          bool inv) {
    typedef typename Rt<C>::R R_;
    const R_ sg = inv ? R_(1) : R_(-1);  // sign of i in w_4 = e^{-+ i pi/2}
    int s0 = 1;
    for (int st = 0; st < nst; ++st) {
        const int R = rad[st];
        const int m = L / (s0 * R);
        const int nb = m * s0;  // butterflies per line
        const int tot = nl * nb;
        for (int b = threadIdx.x; b < tot; b += blockDim.x) {
            const int l = b / nb;
            const int bb = b - l * nb;
            const int p = bb / s0;
            const int q = bb - p * s0;
            const C* xi = x + l * ls + (q + s0 * p) * es;
            C* yo = y + l * ls + (q + s0 * R * p) * es;
            const int tws = p * s0;      // twiddle index step: w_n^{p t} = W[p s t]
            const int ms = m * s0 * es;  // input stride between the radix points
            const int os = s0 * es;      // output stride between the radix points
            if (R == 2) {
                const C a0 = xi[0], a1 = xi[ms];
                yo[0] = cad(a0, a1);
                yo[os] = cml(csb(a0, a1), cwt(W, tws, inv));
            } else if (R == 4) {
                const C a0 = xi[0], a1 = xi[ms], a2 = xi[2 * ms], a3 = xi[3 * ms];
                const C s02 = cad(a0, a2), d02 = csb(a0, a2), s13 = cad(a1, a3), d13 = csb(a1, a3);
                // w_4 = -i (forward): b1 = d02 - i d13, b3 = d02 + i d13
                const C id13 = cis(d13, sg);
                yo[0] = cad(s02, s13);
                yo[os] = cml(cad(d02, id13), cwt(W, tws, inv));
                yo[2 * os] = cml(csb(s02, s13), cwt(W, 2 * tws, inv));
                yo[3 * os] = cml(csb(d02, id13), cwt(W, 3 * tws, inv));
            } else if (R == 3) {
                const C a0 = xi[0], a1 = xi[ms], a2 = xi[2 * ms];
                const C w = cwt(W, L / 3, inv);  // w_3
                const C sm = cad(a1, a2), df = csb(a1, a2);
                const C t = cmk<C>(a0.x + w.x * sm.x, a0.y + w.x * sm.y);
                const C u = cis(df, w.y);  // i Im(w_3) (a1 - a2)
                yo[0] = cad(a0, sm);
                yo[os] = cml(cad(t, u), cwt(W, tws, inv));
                yo[2 * os] = cml(csb(t, u), cwt(W, 2 * tws, inv));
            } else {  // R == 5
                const C a0 = xi[0], a1 = xi[ms], a2 = xi[2 * ms], a3 = xi[3 * ms], a4 = xi[4 * ms];
                const C w1 = cwt(W, L / 5, inv), w2 = cwt(W, 2 * (L / 5), inv);  // w_5, w_5^2
                const C s1 = cad(a1, a4), d1 = csb(a1, a4), s2 = cad(a2, a3), d2 = csb(a2, a3);
                const C ta = cmk<C>(a0.x + w1.x * s1.x + w2.x * s2.x, a0.y + w1.x * s1.y + w2.x * s2.y);
                const C tb = cmk<C>(a0.x + w2.x * s1.x + w1.x * s2.x, a0.y + w2.x * s1.y + w1.x * s2.y);
                // i (Im w1 d1 + Im w2 d2) and i (Im w2 d1 - Im w1 d2)
                const C ua = cmk<C>(-(w1.y * d1.y + w2.y * d2.y), w1.y * d1.x + w2.y * d2.x);
                const C ub = cmk<C>(-(w2.y * d1.y - w1.y * d2.y), w2.y * d1.x - w1.y * d2.x);
                yo[0] = cad(a0, cad(s1, s2));
                yo[os] = cml(cad(ta, ua), cwt(W, tws, inv));
                yo[2 * os] = cml(cad(tb, ub), cwt(W, 2 * tws, inv));
                yo[3 * os] = cml(csb(tb, ub), cwt(W, 3 * tws, inv));
                yo[4 * os] = cml(csb(ta, ua), cwt(W, 4 * tws, inv));
            }
        }
        __syncthreads();
        C* t = x;
        x = y;
        y = t;
        s0 *= R;
    }
    return x;
}

template <typename C>
__device__ __forceinline__ C* fft_lines(C* x, C* y, int nl, int L, const int* rad, int nst, const C* W, bool inv) {
    return fft_lines_s(x, y, nl, L, L, 1, rad, nst, W, inv);
}

template <typename C>
__device__ __forceinline__ void load_tw(C* W, const void* src, int L) {
    const C* w = (const C*)src;
    for (int i = threadIdx.x; i < L; i += blockDim.x) W[i] = w[i];
}

// A: scatter C_G onto the lines of axis 3 and transform them (inverse)
template <typename C>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_a(FftArgs f) {
    extern __shared__ __align__(16) unsigned char fsm[];
    const int F3 = f.F3, LPB = f.lpb[2];
    C* W = (C*)fsm;
    C* x = W + F3;
    C* y = x + LPB * F3;
    const int k = blockIdx.z, c = blockIdx.y;
    const FftK K = f.fk[k];
    const int l0 = blockIdx.x * LPB;
    if (l0 >= K.nline) return;
    const int nl = min(LPB, K.nline - l0);
    load_tw(W, f.w[2], F3);
    for (int i = threadIdx.x; i < nl * F3; i += blockDim.x) x[i] = cmk<C>(0, 0);
    __syncthreads();
    const ToepDesc td = f.td[k];
    const int j0 = K.lg0[l0], j1 = K.lg0[l0 + nl];
    const int base = l0 * F3;
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x)
        x[K.lpos[j] - base] = cvt(td.X[K.gperm[j] + (size_t)c * td.ldx], C());
    __syncthreads();
    const C* r = fft_lines(x, y, nl, F3, f.rad[2], f.nst[2], W, true);
    C* out = (C*)f.b3 + ((size_t)k * f.ncol + c) * f.b3_col + (size_t)base;
    for (int i = threadIdx.x; i < nl * F3; i += blockDim.x) out[i] = r[i];
}

// B (fwd = 0) and D (fwd = 1): axis 2 on the planes holding a G; a block
// takes lpb[1] consecutive r3 of one plane
template <typename C>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_bd(FftArgs f, int fwd) {
    extern __shared__ __align__(16) unsigned char fsm[];
    const int F2 = f.F2, F3 = f.F3, LPB = f.lpb[1];
    C* W = (C*)fsm;
    C* x = W + F2;
    C* y = x + LPB * F2;
    const int k = blockIdx.z, c = blockIdx.y;
    const FftK K = f.fk[k];
    const int nch = (F3 + LPB - 1) / LPB;
    const int p = blockIdx.x / nch, i30 = (blockIdx.x - p * nch) * LPB;
    if (p >= K.nplane) return;
    const int nl = min(LPB, F3 - i30);
    load_tw(W, f.w[1], F2);
    C* b3 = (C*)f.b3 + ((size_t)k * f.ncol + c) * f.b3_col;
    C* b2 = (C*)f.b2 + ((size_t)k * f.ncol + c) * f.b2_col + (size_t)p * F2 * F3;
    const int* lo = K.line_of + (size_t)p * F2;
    for (int i = threadIdx.x; i < F2 * nl; i += blockDim.x) {
        const int r2 = i / nl, l = i - r2 * nl;
        C v = cmk<C>(0, 0);
        if (fwd) {
            v = b2[(size_t)r2 * F3 + i30 + l];
        } else {
            const int id = lo[r2];
            if (id >= 0) v = b3[(size_t)id * F3 + i30 + l];
        }
        x[l * F2 + r2] = v;
    }
    __syncthreads();
    const C* r = fft_lines(x, y, nl, F2, f.rad[1], f.nst[1], W, !fwd);
    for (int i = threadIdx.x; i < F2 * nl; i += blockDim.x) {
        const int r2 = i / nl, l = i - r2 * nl;
        if (fwd) {
            const int id = lo[r2];
            if (id >= 0) b3[(size_t)id * F3 + i30 + l] = r[l * F2 + r2];
        } else {
            b2[(size_t)r2 * F3 + i30 + l] = r[l * F2 + r2];
        }
    }
}

// C: axis 1 on every (r2, r3): inverse, times the potential, forward; the
// result is kept on the planes holding a G
template <typename C>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_c(FftArgs f) {
    extern __shared__ __align__(16) unsigned char fsm[];
    const int F1 = f.F1, F2 = f.F2, F3 = f.F3, LPB = f.lpb[0];
    C* W = (C*)fsm;
    C* x = W + F1;
    C* y = x + LPB * F1;
    const int k = blockIdx.z, c = blockIdx.y;
    const FftK K = f.fk[k];
    const int nch = (F3 + LPB - 1) / LPB;
    const int r2 = blockIdx.x / nch, i30 = (blockIdx.x - r2 * nch) * LPB;
    const int nl = min(LPB, F3 - i30);
    load_tw(W, f.w[0], F1);
    C* b2 = (C*)f.b2 + ((size_t)k * f.ncol + c) * f.b2_col;
    const size_t pst = (size_t)F2 * F3;
    const size_t off = (size_t)r2 * F3 + i30;
    for (int i = threadIdx.x; i < F1 * nl; i += blockDim.x) {
        const int r1 = i / nl, l = i - r1 * nl;
        const int p = K.plane_of[r1];
        x[l * F1 + r1] = (p >= 0) ? b2[(size_t)p * pst + off + l] : cmk<C>(0, 0);
    }
    // the potential of this block's points, loaded (coalesced along r3) before
    // the inverse transform so that the loads overlap it
    constexpr int PV = FFT_PV;  // F1 nl <= FFT_BLK_PTS
    C pv[PV];
    {
        const C* v = (const C*)f.v;
        const C* vd = (const C*)f.vd;
        typedef typename Rt<C>::R R_;
        const R_ sc = f.use_vd ? (R_)(*f.s) : R_(0);
#pragma unroll
        for (int u = 0; u < PV; ++u) {
            const int i = threadIdx.x + u * FFT_THREADS;
            pv[u] = cmk<C>(0, 0);
            if (i < F1 * nl) {
                const int r1 = i / nl, l = i - r1 * nl;
                const size_t gi = (size_t)r1 * pst + off + l;
                if (f.vmode == 0) {
                    pv[u] = v[gi];
                    if (f.use_vd) {
                        const C d = vd[gi];
                        pv[u] = cmk<C>(pv[u].x + sc * d.x, pv[u].y + sc * d.y);
                    }
                } else {
                    const C d = vd[gi];
                    pv[u] = cmk<C>(sc * d.x, sc * d.y);
                }
            }
        }
    }
    __syncthreads();
    C* r = fft_lines(x, y, nl, F1, f.rad[0], f.nst[0], W, true);
#pragma unroll
    for (int u = 0; u < PV; ++u) {
        const int i = threadIdx.x + u * FFT_THREADS;
        if (i < F1 * nl) {
            const int r1 = i / nl, l = i - r1 * nl;
            r[l * F1 + r1] = cml(r[l * F1 + r1], pv[u]);
        }
    }
    __syncthreads();
    const C* o = fft_lines(r, r == x ? y : x, nl, F1, f.rad[0], f.nst[0], W, false);
    for (int i = threadIdx.x; i < F1 * nl; i += blockDim.x) {
        const int r1 = i / nl, l = i - r1 * nl;
        const int p = K.plane_of[r1];
        if (p >= 0) b2[(size_t)p * pst + off + l] = o[l * F1 + r1];
    }
}

// E: transform the lines of axis 3 (forward) and gather Y_G
template <typename C>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_e(FftArgs f) {
    extern __shared__ __align__(16) unsigned char fsm[];
    const int F3 = f.F3, LPB = f.lpb[2];
    C* W = (C*)fsm;
    C* x = W + F3;
    C* y = x + LPB * F3;
    const int k = blockIdx.z, c = blockIdx.y;
    const FftK K = f.fk[k];
    const int l0 = blockIdx.x * LPB;
    if (l0 >= K.nline) return;
    const int nl = min(LPB, K.nline - l0);
    load_tw(W, f.w[2], F3);
    const int base = l0 * F3;
    const C* in = (const C*)f.b3 + ((size_t)k * f.ncol + c) * f.b3_col + (size_t)base;
    for (int i = threadIdx.x; i < nl * F3; i += blockDim.x) x[i] = in[i];
    __syncthreads();
    const C* r = fft_lines(x, y, nl, F3, f.rad[2], f.nst[2], W, false);
    const ToepDesc td = f.td[k];
    const int j0 = K.lg0[l0], j1 = K.lg0[l0 + nl];
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x)
        td.Y[K.gperm[j] + (size_t)c * td.ldy] = todz(r[K.lpos[j] - base]);
}

// A+B (fwd = 0) and D+E (fwd = 1) for one plane holding a G: the plane's
// lines (compacted) along axis 3 and its F3 columns along axis 2, with the
// whole plane in shared memory
template <typename C>
__global__ void __launch_bounds__(FFT_PTHREADS) k_fft_plane(FftArgs f, int fwd) {
    extern __shared__ __align__(16) unsigned char fsm[];
    const int F2 = f.F2, F3 = f.F3, n2 = F2 * F3;
    C* W2 = (C*)fsm;
    C* W3 = W2 + F2;
    C* A = W3 + F3;
    C* B = A + n2;
    const int k = blockIdx.z, c = blockIdx.y, p = blockIdx.x;
    const FftK K = f.fk[k];
    if (p >= K.nplane) return;
    load_tw(W2, f.w[1], F2);
    load_tw(W3, f.w[2], F3);
    const int l0 = K.pl0[p], nl = K.pl0[p + 1] - l0;
    const int base = l0 * F3;
    C* b2 = (C*)f.b2 + ((size_t)k * f.ncol + c) * f.b2_col + (size_t)p * n2;
    const ToepDesc td = f.td[k];
    const int j0 = K.lg0[l0], j1 = K.lg0[l0 + nl];
    if (!fwd) {
        for (int i = threadIdx.x; i < nl * F3; i += blockDim.x) A[i] = cmk<C>(0, 0);
        __syncthreads();
        for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x)
            A[K.lpos[j] - base] = cvt(td.X[K.gperm[j] + (size_t)c * td.ldx], C());
        __syncthreads();
        C* r = fft_lines(A, B, nl, F3, f.rad[2], f.nst[2], W3, true);
        C* P = (r == A) ? B : A;
        for (int i = threadIdx.x; i < n2; i += blockDim.x) P[i] = cmk<C>(0, 0);
        __syncthreads();
        for (int i = threadIdx.x; i < nl * F3; i += blockDim.x) {
            const int l = i / F3, r3 = i - l * F3;
            P[K.lr2[l0 + l] * F3 + r3] = r[i];
        }
        __syncthreads();
        const C* q = fft_lines_s(P, r, F3, F2, 1, F3, f.rad[1], f.nst[1], W2, true);
        for (int i = threadIdx.x; i < n2; i += blockDim.x) b2[i] = q[i];
    } else {
        for (int i = threadIdx.x; i < n2; i += blockDim.x) A[i] = b2[i];
        __syncthreads();
        C* q = fft_lines_s(A, B, F3, F2, 1, F3, f.rad[1], f.nst[1], W2, false);
        C* o = (q == A) ? B : A;
        for (int i = threadIdx.x; i < nl * F3; i += blockDim.x) {
            const int l = i / F3, r3 = i - l * F3;
            o[i] = q[K.lr2[l0 + l] * F3 + r3];
        }
        __syncthreads();
        const C* r = fft_lines(o, q, nl, F3, f.rad[2], f.nst[2], W3, false);
        for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x)
            td.Y[K.gperm[j] + (size_t)c * td.ldy] = todz(r[K.lpos[j] - base]);
    }
}

// Interstitial density of the propagated states on the grid: for every
// (r2, r3) line of axis 1 the inverse transform of each (k, state) column
// (planes from the plane pass), |psi|^2 summed with the weights w_k f_j in
// (k, j) order; n(r) = that sum / Omega (psi~ = sqrt(Omega) psi here)
template <typename C>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_density(FftArgs f, int nk, const double* __restrict__ occ,
                                                          const double* __restrict__ wk, double inv_omega, C* rho) {
    extern __shared__ __align__(16) unsigned char fsm[];
    const int F1 = f.F1, F2 = f.F2, F3 = f.F3, LPB = f.lpb[0];
    C* W = (C*)fsm;
    C* x = W + F1;
    C* y = x + LPB * F1;
    const int nch = (F3 + LPB - 1) / LPB;
    const int r2 = blockIdx.x / nch, i30 = (blockIdx.x - r2 * nch) * LPB;
    const int nl = min(LPB, F3 - i30);
    load_tw(W, f.w[0], F1);
    const size_t pst = (size_t)F2 * F3;
    const size_t off = (size_t)r2 * F3 + i30;
    constexpr int PV = FFT_PV;
    double acc[PV];
#pragma unroll
    for (int u = 0; u < PV; ++u) acc[u] = 0.0;
    for (int k = 0; k < nk; ++k) {
        const FftK K = f.fk[k];
        for (int c = 0; c < f.ncol; ++c) {
            const C* b2 = (const C*)f.b2 + ((size_t)k * f.ncol + c) * f.b2_col;
            for (int i = threadIdx.x; i < F1 * nl; i += blockDim.x) {
                const int r1 = i / nl, l = i - r1 * nl;
                const int p = K.plane_of[r1];
                x[l * F1 + r1] = (p >= 0) ? b2[(size_t)p * pst + off + l] : cmk<C>(0, 0);
            }
            __syncthreads();
            const C* r = fft_lines(x, y, nl, F1, f.rad[0], f.nst[0], W, true);
            const double wf = wk[k] * occ[c];
#pragma unroll
            for (int u = 0; u < PV; ++u) {
                const int i = threadIdx.x + u * FFT_THREADS;
                if (i < F1 * nl) {
                    const int r1 = i / nl, l = i - r1 * nl;
                    const C v = r[l * F1 + r1];
                    acc[u] += wf * ((double)v.x * v.x + (double)v.y * v.y);
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int u = 0; u < PV; ++u) {
        const int i = threadIdx.x + u * FFT_THREADS;
        if (i < F1 * nl) {
            const int r1 = i / nl, l = i - r1 * nl;
            rho[(size_t)r1 * pst + off + l] = cmk<C>((typename Rt<C>::R)(acc[u] * inv_omega), 0);
        }
    }
}

// A full-grid 1-D pass along `axis` (0, 1, 2) in place, every line
template <typename C>
__global__ void __launch_bounds__(FFT_THREADS) k_fft_full(FftArgs f, C* buf, int axis, int inv) {
    extern __shared__ __align__(16) unsigned char fsm[];
    const int F1 = f.F1, F2 = f.F2, F3 = f.F3;
    const int L = axis == 0 ? F1 : (axis == 1 ? F2 : F3);
    const int LPB = f.lpb[axis];
    C* W = (C*)fsm;
    C* x = W + L;
    C* y = x + LPB * L;
    load_tw(W, f.w[axis], L);
    size_t base, es, ls;
    int nl;
    if (axis == 2) {
        const int l0 = blockIdx.x * LPB;
        nl = min(LPB, F1 * F2 - l0);
        base = (size_t)l0 * F3;
        es = 1;
        ls = F3;
    } else {
        const int nch = (F3 + LPB - 1) / LPB;
        const int o = blockIdx.x / nch, i30 = (blockIdx.x - o * nch) * LPB;
        nl = min(LPB, F3 - i30);
        es = axis == 1 ? (size_t)F3 : (size_t)F2 * F3;
        base = (axis == 1 ? (size_t)o * F2 * F3 : (size_t)o * F3) + i30;
        ls = 1;
    }
    // element j of line l at base + l ls + j es; coalesced along l for axes 0, 1
    for (int i = threadIdx.x; i < nl * L; i += blockDim.x) {
        int l, j;
        if (axis == 2) {
            l = i / L;
            j = i - l * L;
        } else {
            j = i / nl;
            l = i - j * nl;
        }
        x[l * L + j] = buf[base + l * ls + j * es];
    }
    __syncthreads();
    const C* r = fft_lines(x, y, nl, L, f.rad[axis], f.nst[axis], W, inv != 0);
    for (int i = threadIdx.x; i < nl * L; i += blockDim.x) {
        int l, j;
        if (axis == 2) {
            l = i / L;
            j = i - l * L;
        } else {
            j = i / nl;
            l = i - j * nl;
        }
        buf[base + l * ls + j * es] = r[l * L + j];
    }
}

// Poisson equation on the table box: vd(g) = 4 pi (N - N0)(g) / (F^6 |g|^2)
// at the residues of |g_i| <= e_i, g != 0, zero elsewhere (N = F^3 n_g; the
// second F^3 is the normalisation of the potential's grid image), and the sum
// of |dV_g| for the bound check
template <typename C>
__global__ void k_hartree(const C* __restrict__ N, const C* __restrict__ N0, C* vd, int F1, int F2, int F3, int e0,
                          int e1, int e2, double b00, double b01, double b02, double b10, double b11, double b12,
                          double b20, double b21, double b22, double inv_f3, double* l1) {
    __shared__ double part[8];
    const size_t n = (size_t)F1 * F2 * F3;
    double mine = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int r2 = (int)(i % F3), r1 = (int)((i / F3) % F2), r0 = (int)(i / ((size_t)F2 * F3));
        const int d0 = r0 <= e0 ? r0 : (r0 >= F1 - e0 ? r0 - F1 : 1 << 20);
        const int d1 = r1 <= e1 ? r1 : (r1 >= F2 - e1 ? r1 - F2 : 1 << 20);
        const int d2 = r2 <= e2 ? r2 : (r2 >= F3 - e2 ? r2 - F3 : 1 << 20);
        C out = cmk<C>(0, 0);
        if (d0 != (1 << 20) && d1 != (1 << 20) && d2 != (1 << 20) && (d0 | d1 | d2) != 0) {
            const double gx = d0 * b00 + d1 * b10 + d2 * b20;
            const double gy = d0 * b01 + d1 * b11 + d2 * b21;
            const double gz = d0 * b02 + d1 * b12 + d2 * b22;
            const double g2 = gx * gx + gy * gy + gz * gz;
            const double f = 4.0 * 3.14159265358979323846 * inv_f3 / g2;  // 4 pi / (F^3 |g|^2)
            const double dre = ((double)N[i].x - (double)N0[i].x) * inv_f3;
            const double dim = ((double)N[i].y - (double)N0[i].y) * inv_f3;
            out = cmk<C>((typename Rt<C>::R)(f * dre), (typename Rt<C>::R)(f * dim));
            mine += f * sqrt(dre * dre + dim * dim) / inv_f3;
        }
        vd[i] = out;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    mine = warp_sum(mine);
    if (lane == 0) part[warp] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        atomicAdd(l1, t);  // only compared with the bound: the order does not matter
    }
}

// the device accumulator compared with the bound after every step (other parts of
// the potential change add their own bounds to it before the check)
double* fft_l1(const FftPlan* pl) { return pl ? pl->l1 : nullptr; }

// the l1 norm of dV against the bound of the spectral interval; flag bit 6
__global__ void k_hartree_check(double* l1, double bound, int* flag) {
    if (*l1 > bound) atomicOr(flag, 64);
    *l1 = 0.0;
}

// ---------------------------------------------------------------- set-up kernels
// V~ placed on the grid by residue
__global__ void k_fft_place(const zd* tab, int d0, int d1, int d2, int F1, int F2, int F3, zd* grid) {
    const int n = d0 * d1 * d2;
    const int e0 = (d0 - 1) / 2, e1 = (d1 - 1) / 2, e2 = (d2 - 1) / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int i2 = i % d2, i1 = (i / d2) % d1, i0 = i / (d1 * d2);
        const int r0 = ((i0 - e0) % F1 + F1) % F1;
        const int r1 = ((i1 - e1) % F2 + F2) % F2;
        const int r2 = ((i2 - e2) % F3 + F3) % F3;
        grid[((size_t)r0 * F2 + r1) * F3 + r2] = tab[i];
    }
}

// out = scale * (inverse DFT along axis `ax` of in), directly (set-up only)
__global__ void k_fft_dft_axis(const zd* in, zd* out, int F1, int F2, int F3, int ax, const zd* W, double scale) {
    const int n = F1 * F2 * F3;
    const int L = ax == 0 ? F1 : (ax == 1 ? F2 : F3);
    const int st = ax == 0 ? F2 * F3 : (ax == 1 ? F3 : 1);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int j = (i / st) % L;
        const int b = i - j * st;
        zd acc = zmk(0.0, 0.0);
        for (int m = 0; m < L; ++m) {
            const zd w = W[(int)(((long long)j * m) % L)];
            zfma(acc, in[b + (size_t)m * st], zmk(w.x, -w.y));
        }
        out[i] = zscale(acc, scale);
    }
}

__global__ void k_fft_to32(const zd* in, zf* out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

// ---------------------------------------------------------------- host side
static bool factor_axis(int n, int* rad, int* nst) {
    int k = 0;
    while (n % 4 == 0 && k < FFT_MAX_ST) {
        rad[k++] = 4;
        n /= 4;
    }
    const int ps[3] = {2, 3, 5};
    for (int pi = 0; pi < 3; ++pi)
        while (n % ps[pi] == 0 && k < FFT_MAX_ST) {
            rad[k++] = ps[pi];
            n /= ps[pi];
        }
    *nst = k;
    return n == 1;
}

// smallest 2^a 3^b 5^c >= n
static int smooth_at_least(int n) {
    for (int m = std::max(n, 1);; ++m) {
        int r = m;
        for (int p : {2, 3, 5})
            while (r % p == 0) r /= p;
        if (r == 1) return m;
    }
}

static size_t fft_smem(int L, int elt) { return (size_t)(L + 2 * fft_lpb(L) * L) * elt; }
static size_t fft_plane_smem(int F2, int F3, int elt) { return (size_t)(F2 + F3 + 2 * F2 * F3) * elt; }
#define FFT_PLANE_SMEM_MAX (200 * 1024)

template <typename T> static T* fdalloc(size_t n, std::string* why, bool* ok) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
        *ok = false;
        if (why) *why = "FFT route: device allocation failed";
        return nullptr;
    }
    return (T*)p;
}

int fft_grid_for(const int vt_dim[3], int F[3]) {
    for (int i = 0; i < 3; ++i) {
        F[i] = smooth_at_least(vt_dim[i]);
        if (F[i] > FFT_MAX_N) return -1;
    }
    return 0;
}

static bool potential_on_grid(const FftPlan* pl, const zd* tab, const int vt_dim[3], zd* v64, zf* v32,
                              cudaStream_t st) {
    const int F1 = pl->F[0], F2 = pl->F[1], F3 = pl->F[2];
    const size_t n = (size_t)F1 * F2 * F3;
    zd* tmp = nullptr;
    if (cudaMalloc(&tmp, n * sizeof(zd)) != cudaSuccess) return false;
    cudaMemsetAsync(v64, 0, n * sizeof(zd), st);
    k_fft_place<<<256, 256, 0, st>>>(tab, vt_dim[0], vt_dim[1], vt_dim[2], F1, F2, F3, v64);
    const double inv = 1.0 / ((double)F1 * F2 * F3);
    const int nb = (int)std::min<size_t>((n + 255) / 256, 4096);
    k_fft_dft_axis<<<nb, 256, 0, st>>>(v64, tmp, F1, F2, F3, 0, pl->w64[0], 1.0);
    k_fft_dft_axis<<<nb, 256, 0, st>>>(tmp, v64, F1, F2, F3, 1, pl->w64[1], 1.0);
    cudaMemcpyAsync(tmp, v64, n * sizeof(zd), cudaMemcpyDeviceToDevice, st);
    k_fft_dft_axis<<<nb, 256, 0, st>>>(tmp, v64, F1, F2, F3, 2, pl->w64[2], inv);
    if (v32) k_fft_to32<<<nb, 256, 0, st>>>(v64, v32, n);
    const bool ok = cudaStreamSynchronize(st) == cudaSuccess;
    cudaFree(tmp);
    return ok;
}

static bool fft_alloc_buffers(FftPlan* pl, int ncol, std::string* why) {
    const size_t elt = pl->prec == 0 ? sizeof(zd) : sizeof(zf);
    const size_t c3 = (size_t)pl->max_lines * pl->F[2];
    const size_t c2 = (size_t)pl->max_planes * pl->F[1] * pl->F[2];
    void* b3 = nullptr;
    void* b2 = nullptr;
    if (cudaMalloc(&b3, std::max<size_t>((size_t)pl->nk * ncol * c3 * elt, 16)) != cudaSuccess ||
        cudaMalloc(&b2, std::max<size_t>((size_t)pl->nk * ncol * c2 * elt, 16)) != cudaSuccess) {
        if (b3) cudaFree(b3);
        if (why) *why = "FFT route: device allocation of the transform buffers failed";
        return false;
    }
    if (pl->b3) cudaFree(pl->b3);
    if (pl->b2) cudaFree(pl->b2);
    pl->b3 = b3;
    pl->b2 = b2;
    pl->ncol = ncol;
    return true;
}

int fft_plan_create(FftPlan** out, int nk, const int* ng, const int* const* gint, const int vt_dim[3],
                    const zd* vtab_dev, int ncol, int prec, cudaStream_t st, std::string* why) {
    *out = nullptr;
    FftPlan* pl = new FftPlan();
    pl->prec = prec;
    pl->nk = nk;
    if (fft_grid_for(vt_dim, pl->F)) {
        if (why) *why = "FFT route: a table extent needs more than 512 grid points";
        delete pl;
        return RTTDDFT_ERR_UNSUPPORTED;
    }
    for (int a = 0; a < 3; ++a) factor_axis(pl->F[a], pl->rad[a], &pl->nst[a]);
    bool ok = true;
    // twiddles from the C library's cos and sin in FP64
    for (int a = 0; a < 3; ++a) {
        const int L = pl->F[a];
        std::vector<zd> w(L);
        std::vector<zf> w32(L);
        for (int m = 0; m < L; ++m) {
            const double ang = 2.0 * M_PI * (double)m / (double)L;
            w[m] = zmk(std::cos(ang), -std::sin(ang));
            w32[m] = make_float2((float)w[m].x, (float)w[m].y);
        }
        pl->w64[a] = fdalloc<zd>(L, why, &ok);
        pl->w32[a] = fdalloc<zf>(L, why, &ok);
        if (!ok) break;
        cudaMemcpy(pl->w64[a], w.data(), L * sizeof(zd), cudaMemcpyHostToDevice);
        cudaMemcpy(pl->w32[a], w32.data(), L * sizeof(zf), cudaMemcpyHostToDevice);
    }
    // per-k line tables: entries sorted by (n1, n2, n3); a line is a run of
    // equal (n1, n2), a plane a run of equal n1
    const int F1 = pl->F[0], F2 = pl->F[1], F3 = pl->F[2];
    std::vector<FftK> hk(nk);
    pl->max_lines = 1;
    pl->max_planes = 1;
    for (int k = 0; k < nk && ok; ++k) {
        const int n = ng[k];
        const int* gi = gint[k];
        std::vector<int> perm(n);
        for (int g = 0; g < n; ++g) perm[g] = g;
        std::sort(perm.begin(), perm.end(), [&](int a, int b) {
            const int* x = gi + 3 * a;
            const int* y = gi + 3 * b;
            if (x[0] != y[0]) return x[0] < y[0];
            if (x[1] != y[1]) return x[1] < y[1];
            return x[2] < y[2];
        });
        auto res = [](int v, int F) { return ((v % F) + F) % F; };
        std::vector<int> lg0, lpos(n), plane_of(F1, -1), line_of, pl0, lr2;
        int nline = 0, nplane = 0;
        for (int j = 0; j < n; ++j) {
            const int* t = gi + 3 * perm[j];
            const bool newplane = (j == 0) || t[0] != gi[3 * perm[j - 1]];
            const bool newline = newplane || t[1] != gi[3 * perm[j - 1] + 1];
            if (newplane) {
                plane_of[res(t[0], F1)] = nplane++;
                line_of.resize((size_t)nplane * F2, -1);
                pl0.push_back(nline);
            }
            if (newline) {
                lg0.push_back(j);
                lr2.push_back(res(t[1], F2));
                line_of[(size_t)(nplane - 1) * F2 + res(t[1], F2)] = nline++;
            }
            lpos[j] = (nline - 1) * F3 + res(t[2], F3);
        }
        lg0.push_back(n);
        pl0.push_back(nline);
        auto up = [&](const std::vector<int>& v) -> const int* {
            int* d = fdalloc<int>(v.size(), why, &ok);
            if (!ok) return nullptr;
            cudaMemcpy(d, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice);
            pl->tables.push_back(d);
            return d;
        };
        hk[k].nline = nline;
        hk[k].nplane = nplane;
        hk[k].lg0 = up(lg0);
        hk[k].gperm = up(perm);
        hk[k].lpos = up(lpos);
        hk[k].plane_of = up(plane_of);
        hk[k].line_of = up(line_of);
        hk[k].pl0 = up(pl0);
        hk[k].lr2 = up(lr2);
        pl->max_lines = std::max(pl->max_lines, nline);
        pl->max_planes = std::max(pl->max_planes, nplane);
    }
    if (ok) {
        pl->d_fk = fdalloc<FftK>(nk, why, &ok);
        if (ok) cudaMemcpy(pl->d_fk, hk.data(), nk * sizeof(FftK), cudaMemcpyHostToDevice);
    }
    const size_t n3 = (size_t)F1 * F2 * F3;
    if (ok) pl->v64 = fdalloc<zd>(n3, why, &ok);
    if (ok && prec != 0) pl->v32 = fdalloc<zf>(n3, why, &ok);
    if (ok) ok = fft_alloc_buffers(pl, ncol, why);
    if (ok && !potential_on_grid(pl, vtab_dev, vt_dim, pl->v64, pl->v32, st)) {
        ok = false;
        if (why) *why = "FFT route: the potential's grid image failed";
    }
    if (ok) {
        // dynamic shared memory beyond 48 KB for the longest axes
        const int elt = prec == 0 ? (int)sizeof(zd) : (int)sizeof(zf);
        const int mx = (int)fft_smem(std::max(F1, std::max(F2, F3)), elt);
        const size_t psm = fft_plane_smem(F2, F3, elt);
        if (psm <= FFT_PLANE_SMEM_MAX) {
            if (prec == 0) cudaFuncSetAttribute(k_fft_plane<zd>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm);
            else cudaFuncSetAttribute(k_fft_plane<zf>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm);
        }
        if (prec == 0) {
            cudaFuncSetAttribute(k_fft_a<zd>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
            cudaFuncSetAttribute(k_fft_bd<zd>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
            cudaFuncSetAttribute(k_fft_c<zd>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
            cudaFuncSetAttribute(k_fft_e<zd>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        } else {
            cudaFuncSetAttribute(k_fft_a<zf>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
            cudaFuncSetAttribute(k_fft_bd<zf>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
            cudaFuncSetAttribute(k_fft_c<zf>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
            cudaFuncSetAttribute(k_fft_e<zf>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        }
        if (cudaGetLastError() != cudaSuccess) {
            ok = false;
            if (why) *why = "FFT route: set-up kernels failed";
        }
    }
    if (!ok) {
        fft_plan_destroy(pl);
        return RTTDDFT_ERR_OOM;
    }
    *out = pl;
    return 0;
}

int fft_set_dv(FftPlan* pl, const zd* dvtab_dev, const int vt_dim[3], int ncol, cudaStream_t st,
               std::string* why) {
    const size_t n3 = (size_t)pl->F[0] * pl->F[1] * pl->F[2];
    bool ok = true;
    if (!pl->vd64) pl->vd64 = fdalloc<zd>(n3, why, &ok);
    if (ok && pl->prec != 0 && !pl->vd32) pl->vd32 = fdalloc<zf>(n3, why, &ok);
    if (!ok) return RTTDDFT_ERR_OOM;
    if (ncol > pl->ncol) {
        cudaStreamSynchronize(st);
        if (!fft_alloc_buffers(pl, ncol, why)) return RTTDDFT_ERR_OOM;
    }
    if (!potential_on_grid(pl, dvtab_dev, vt_dim, pl->vd64, pl->vd32, st) || cudaGetLastError() != cudaSuccess) {
        if (why) *why = "FFT route: potential change set-up failed";
        return RTTDDFT_ERR_CUDA;
    }
    return 0;
}

// transform buffers for at least ncol columns per k-point
int fft_reserve_columns(FftPlan* pl, int ncol, cudaStream_t st, std::string* why) {
    if (ncol <= pl->ncol) return 0;
    cudaStreamSynchronize(st);
    return fft_alloc_buffers(pl, ncol, why) ? 0 : RTTDDFT_ERR_OOM;
}

void fft_plan_destroy(FftPlan* pl) {
    if (!pl) return;
    for (int a = 0; a < 3; ++a) {
        if (pl->w64[a]) cudaFree(pl->w64[a]);
        if (pl->w32[a]) cudaFree(pl->w32[a]);
    }
    for (void* p : {(void*)pl->v64, (void*)pl->v32, (void*)pl->vd64, (void*)pl->vd32, (void*)pl->d_fk, pl->b3, pl->b2,
                    (void*)pl->rho, (void*)pl->rho0, (void*)pl->l1, (void*)pl->b3d, (void*)pl->b2d})
        if (p) cudaFree(p);
    for (void* p : pl->tables) cudaFree(p);
    delete pl;
}

void fft_plan_info(const FftPlan* pl, int F[3], int* fused) {
    for (int a = 0; a < 3; ++a) F[a] = pl ? pl->F[a] : 0;
    if (fused) *fused = pl ? pl->fused : 0;
}

// The convolution for k-points kofs .. kofs + nk - 1 (descriptors td[kofs ..])
// over ncol columns; vmode 0 multiplies by v (+ s vd when
// use_vd), vmode 1 by s vd alone.  Five launches.
static int launch_fft_any(const FftPlan* pl, int fused, const ToepDesc* td, int kofs, int nk, int ncol, int vmode,
                          int use_vd, const double* s, cudaStream_t st) {
    FftArgs f;
    f.F1 = pl->F[0];
    f.F2 = pl->F[1];
    f.F3 = pl->F[2];
    for (int a = 0; a < 3; ++a) {
        f.nst[a] = pl->nst[a];
        for (int i = 0; i < FFT_MAX_ST; ++i) f.rad[a][i] = pl->rad[a][i];
        f.lpb[a] = fft_lpb(pl->F[a]);
        f.w[a] = pl->prec == 0 ? (const void*)pl->w64[a] : (const void*)pl->w32[a];
    }
    f.fk = pl->d_fk + kofs;
    f.td = td + kofs;
    f.b3 = pl->b3;
    f.b2 = pl->b2;
    f.b3_col = (size_t)pl->max_lines * f.F3;
    f.b2_col = (size_t)pl->max_planes * f.F2 * f.F3;
    f.ncol = ncol;
    f.vmode = vmode;
    f.use_vd = use_vd;
    f.v = pl->prec == 0 ? (const void*)pl->v64 : (const void*)pl->v32;
    f.vd = pl->prec == 0 ? (const void*)pl->vd64 : (const void*)pl->vd32;
    f.s = s;
    const int ch1 = (f.F3 + f.lpb[1] - 1) / f.lpb[1], ch0 = (f.F3 + f.lpb[0] - 1) / f.lpb[0];
    const dim3 ga((pl->max_lines + f.lpb[2] - 1) / f.lpb[2], ncol, nk);
    const dim3 gb(pl->max_planes * ch1, ncol, nk);
    const dim3 gc(f.F2 * ch0, ncol, nk);
    if (fused) {
        const dim3 gp(pl->max_planes, ncol, nk);
        if (pl->prec == 0) {
            const size_t psm = fft_plane_smem(f.F2, f.F3, sizeof(zd));
            k_fft_plane<zd><<<gp, FFT_PTHREADS, psm, st>>>(f, 0);
            k_fft_c<zd><<<gc, FFT_THREADS, fft_smem(f.F1, sizeof(zd)), st>>>(f);
            k_fft_plane<zd><<<gp, FFT_PTHREADS, psm, st>>>(f, 1);
        } else {
            const size_t psm = fft_plane_smem(f.F2, f.F3, sizeof(zf));
            k_fft_plane<zf><<<gp, FFT_PTHREADS, psm, st>>>(f, 0);
            k_fft_c<zf><<<gc, FFT_THREADS, fft_smem(f.F1, sizeof(zf)), st>>>(f);
            k_fft_plane<zf><<<gp, FFT_PTHREADS, psm, st>>>(f, 1);
        }
        return 3;
    }
    if (pl->prec == 0) {
        k_fft_a<zd><<<ga, FFT_THREADS, fft_smem(f.F3, sizeof(zd)), st>>>(f);
        k_fft_bd<zd><<<gb, FFT_THREADS, fft_smem(f.F2, sizeof(zd)), st>>>(f, 0);
        k_fft_c<zd><<<gc, FFT_THREADS, fft_smem(f.F1, sizeof(zd)), st>>>(f);
        k_fft_bd<zd><<<gb, FFT_THREADS, fft_smem(f.F2, sizeof(zd)), st>>>(f, 1);
        k_fft_e<zd><<<ga, FFT_THREADS, fft_smem(f.F3, sizeof(zd)), st>>>(f);
    } else {
        k_fft_a<zf><<<ga, FFT_THREADS, fft_smem(f.F3, sizeof(zf)), st>>>(f);
        k_fft_bd<zf><<<gb, FFT_THREADS, fft_smem(f.F2, sizeof(zf)), st>>>(f, 0);
        k_fft_c<zf><<<gc, FFT_THREADS, fft_smem(f.F1, sizeof(zf)), st>>>(f);
        k_fft_bd<zf><<<gb, FFT_THREADS, fft_smem(f.F2, sizeof(zf)), st>>>(f, 1);
        k_fft_e<zf><<<ga, FFT_THREADS, fft_smem(f.F3, sizeof(zf)), st>>>(f);
    }
    return 5;
}

int launch_fft_conv(const FftPlan* pl, const ToepDesc* td, int kofs, int nk, int ncol, int vmode, int use_vd,
                    const double* s, cudaStream_t st) {
    return launch_fft_any(pl, pl->fused, td, kofs, nk, ncol, vmode, use_vd, s, st);
}

// Set-up autotuner: times the five-launch and the plane-fused three-launch
// sets on the operator's own descriptors (three runs each after one warm-up)
// and keeps the faster.
// RTTDDFT_FFT_LAUNCHES=5 or =3 in the environment fixes the choice (both sets
// compute the same sums; the tests run each).
int fft_tune(FftPlan* pl, const ToepDesc* td, int ncol, cudaStream_t st) {
    const int elt = pl->prec == 0 ? (int)sizeof(zd) : (int)sizeof(zf);
    if (fft_plane_smem(pl->F[1], pl->F[2], elt) > FFT_PLANE_SMEM_MAX) {
        pl->fused = 0;
        return 0;
    }
    const char* force = getenv("RTTDDFT_FFT_LAUNCHES");
    if (force && (force[0] == '3' || force[0] == '5') && force[1] == 0) {
        pl->fused = force[0] == '3' ? 1 : 0;
        return 0;
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -1;
    }
    float ms[2] = {0.f, 0.f};
    for (int v = 0; v < 2; ++v) {
        launch_fft_any(pl, v, td, 0, pl->nk, ncol, 0, 0, nullptr, st);
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3; ++r) launch_fft_any(pl, v, td, 0, pl->nk, ncol, 0, 0, nullptr, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms[v], e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pl->ms_split = ms[0] / 3;
    pl->ms_fused = ms[1] / 3;
    pl->fused = ms[1] < ms[0] ? 1 : 0;
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------------- Hartree feedback
// launch arguments of the FP64 density passes
static FftArgs fft_args64(const FftPlan* pl, const ToepDesc* td, int kofs, int ncol) {
    FftArgs f;
    f.F1 = pl->F[0];
    f.F2 = pl->F[1];
    f.F3 = pl->F[2];
    for (int a = 0; a < 3; ++a) {
        f.nst[a] = pl->nst[a];
        for (int i = 0; i < FFT_MAX_ST; ++i) f.rad[a][i] = pl->rad[a][i];
        f.lpb[a] = fft_lpb(pl->F[a]);
        f.w[a] = (const void*)pl->w64[a];
    }
    f.fk = pl->d_fk + kofs;
    f.td = td + kofs;
    f.b3 = pl->prec == 0 ? pl->b3 : (void*)pl->b3d;
    f.b2 = pl->prec == 0 ? pl->b2 : (void*)pl->b2d;
    f.b3_col = (size_t)pl->max_lines * f.F3;
    f.b2_col = (size_t)pl->max_planes * f.F2 * f.F3;
    f.ncol = ncol;
    f.vmode = 0;
    f.use_vd = 0;
    f.v = nullptr;
    f.vd = nullptr;
    f.s = nullptr;
    return f;
}

// Set up the density feedback: grids for n, its starting value and the
// potential change; recip rows are the reciprocal vectors b_i (1/bohr).
int fft_hartree_init(FftPlan* pl, const double recip[9], const int vt_dim[3], double omega, double bound, int ns,
                     cudaStream_t st, std::string* why) {
    const size_t n3 = (size_t)pl->F[0] * pl->F[1] * pl->F[2];
    bool ok = true;
    if (cudaMalloc((void**)&pl->rho, n3 * sizeof(zd)) != cudaSuccess ||
        cudaMalloc((void**)&pl->rho0, n3 * sizeof(zd)) != cudaSuccess ||
        cudaMalloc((void**)&pl->l1, sizeof(double)) != cudaSuccess)
        ok = false;
    if (ok && !pl->vd64) ok = cudaMalloc((void**)&pl->vd64, n3 * sizeof(zd)) == cudaSuccess;
    if (ok && pl->prec != 0 && !pl->vd32) ok = cudaMalloc((void**)&pl->vd32, n3 * sizeof(zf)) == cudaSuccess;
    if (ok && pl->prec != 0) {
        // FP64 buffers for the N_s columns of the density
        const size_t c3 = (size_t)pl->max_lines * pl->F[2], c2 = (size_t)pl->max_planes * pl->F[1] * pl->F[2];
        ok = cudaMalloc((void**)&pl->b3d, std::max<size_t>((size_t)pl->nk * ns * c3, 1) * sizeof(zd)) == cudaSuccess &&
             cudaMalloc((void**)&pl->b2d, std::max<size_t>((size_t)pl->nk * ns * c2, 1) * sizeof(zd)) == cudaSuccess;
    }
    if (!ok) {
        if (why) *why = "Hartree feedback: device allocation failed";
        return RTTDDFT_ERR_OOM;
    }
    cudaMemsetAsync(pl->l1, 0, sizeof(double), st);
    cudaMemsetAsync(pl->vd64, 0, n3 * sizeof(zd), st);
    if (pl->vd32) cudaMemsetAsync(pl->vd32, 0, n3 * sizeof(zf), st);
    const size_t psm = fft_plane_smem(pl->F[1], pl->F[2], sizeof(zd));
    pl->fused_d = (pl->prec == 0) ? pl->fused : (psm <= FFT_PLANE_SMEM_MAX ? 1 : 0);
    for (int i = 0; i < 9; ++i) pl->recip[i] = recip[i];
    for (int a = 0; a < 3; ++a) pl->e[a] = (vt_dim[a] - 1) / 2;
    pl->omega = omega;
    pl->bound = bound;
    pl->hartree = 1;
    const int mx = (int)fft_smem(std::max(pl->F[0], std::max(pl->F[1], pl->F[2])), (int)sizeof(zd));
    cudaFuncSetAttribute(k_fft_density<zd>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_fft_full<zd>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_fft_a<zd>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_fft_bd<zd>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (pl->fused_d) cudaFuncSetAttribute(k_fft_plane<zd>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm);
    if (cudaGetLastError() != cudaSuccess) {
        if (why) *why = "Hartree feedback: set-up failed";
        return RTTDDFT_ERR_CUDA;
    }
    return 0;
}

template <typename C>
static int density_launches(const FftPlan* pl, const FftArgs& f, int nk, const double* occ, const double* wk, C* rho,
                            cudaStream_t st) {
    const int ch0 = (f.F3 + f.lpb[0] - 1) / f.lpb[0], ch1 = (f.F3 + f.lpb[1] - 1) / f.lpb[1];
    int nl = 0;
    // the planes of every (k, state) column after the inverse transforms of axes 3 and 2
    if (pl->fused_d) {
        k_fft_plane<C><<<dim3(pl->max_planes, f.ncol, nk), FFT_PTHREADS, fft_plane_smem(f.F2, f.F3, sizeof(C)), st>>>(f, 0);
        ++nl;
    } else {
        k_fft_a<C><<<dim3((pl->max_lines + f.lpb[2] - 1) / f.lpb[2], f.ncol, nk), FFT_THREADS,
                     fft_smem(f.F3, sizeof(C)), st>>>(f);
        k_fft_bd<C><<<dim3(pl->max_planes * ch1, f.ncol, nk), FFT_THREADS, fft_smem(f.F2, sizeof(C)), st>>>(f, 0);
        nl += 2;
    }
    k_fft_density<C><<<f.F2 * ch0, FFT_THREADS, fft_smem(f.F1, sizeof(C)), st>>>(f, nk, occ, wk, 1.0 / pl->omega, rho);
    ++nl;
    // N(g) = sum_r n(r) e^{-2 pi i g.r/F}
    const int ga[3] = {f.F2 * ch0, f.F1 * ch1, (f.F1 * f.F2 + f.lpb[2] - 1) / f.lpb[2]};
    for (int a = 2; a >= 0; --a) {
        const int L = pl->F[a];
        k_fft_full<C><<<ga[a], FFT_THREADS, fft_smem(L, sizeof(C)), st>>>(f, rho, a, 0);
        ++nl;
    }
    return nl;
}

// The density of the current C (td: per k {C, .}) transformed to G space; with
// reference = 1 it becomes the starting density n(0).  Returns the launches.
int launch_fft_density(const FftPlan* pl, const ToepDesc* td, int nk, int ns, const double* occ, const double* wk,
                       int reference, cudaStream_t st) {
    const FftArgs f = fft_args64(pl, td, 0, ns);
    const size_t n3 = (size_t)pl->F[0] * pl->F[1] * pl->F[2];
    const int nl = density_launches<zd>(pl, f, nk, occ, wk, pl->rho, st);
    if (reference) cudaMemcpyAsync(pl->rho0, pl->rho, n3 * sizeof(zd), cudaMemcpyDeviceToDevice, st);
    return nl;
}

// After a step: the density of C_{k+1}, its Hartree potential change against
// n(0) on the table box, and that potential's grid image for the next step's
// operator and potential-change rebuild.  Returns the launches.
int launch_fft_hartree(const FftPlan* pl, const ToepDesc* td, int nk, int ns, const double* occ, const double* wk,
                       int* flag, cudaStream_t st) {
    int nl = launch_fft_density(pl, td, nk, ns, occ, wk, 0, st);
    const FftArgs f = fft_args64(pl, td, 0, ns);
    const double inv_f3 = 1.0 / ((double)pl->F[0] * pl->F[1] * pl->F[2]);
    const double* b = pl->recip;
    const int ch0 = (f.F3 + f.lpb[0] - 1) / f.lpb[0], ch1 = (f.F3 + f.lpb[1] - 1) / f.lpb[1];
    const int ga[3] = {f.F2 * ch0, f.F1 * ch1, (f.F1 * f.F2 + f.lpb[2] - 1) / f.lpb[2]};
    k_hartree<zd><<<152, 256, 0, st>>>(pl->rho, pl->rho0, pl->vd64, f.F1, f.F2, f.F3, pl->e[0], pl->e[1], pl->e[2],
                                       b[0], b[1], b[2], b[3], b[4], b[5], b[6], b[7], b[8], inv_f3, pl->l1);
    for (int a = 0; a < 3; ++a)
        k_fft_full<zd><<<ga[a], FFT_THREADS, fft_smem(pl->F[a], sizeof(zd)), st>>>(f, pl->vd64, a, 1);
    if (pl->prec != 0) {
        // the FP32 operator reads its copy of the grid image
        const size_t n3 = (size_t)f.F1 * f.F2 * f.F3;
        k_fft_to32<<<(int)std::min<size_t>((n3 + 255) / 256, 4096), 256, 0, st>>>(pl->vd64, pl->vd32, n3);
        ++nl;
    }
    k_hartree_check<<<1, 1, 0, st>>>(pl->l1, pl->bound, flag);
    return nl + 5;
}
