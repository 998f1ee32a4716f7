// C ABI of the rttddft library (declarations and contracts in include/rttddft.h).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cstdlib>
#include <complex>
#include <string>
#include <vector>

#include "rtd.h"
#include "rttddft.h"

typedef std::complex<double> cplx;

namespace {
thread_local std::string g_last_error;

struct Fail {
    int code;
};
}  // namespace

struct rttddft_ctx {
    int nk = 0, natoms = 0, ns = 0, naux = 0;
    double omega = 0, c = 0;
    rttddft_options opt{};
    AtomTab at{};
    std::vector<int> ng, nb;
    int maxng = 0, maxnb = 0, maxm = 0;
    int vt_dim[3] = {0, 0, 0};
    int nvt = 0, vt_center = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = -1;  // the device current at set-up: every allocation of the context lives there
    std::vector<void*> allocs;
    std::vector<KDev> hkd;
    KDev* d_kd = nullptr;
    AtomTab* d_at = nullptr;
    zd *d_h = nullptr, *d_o = nullptr, *d_p = nullptr, *d_dh = nullptr;
    zf *d_h32 = nullptr, *d_o32 = nullptr, *d_p32 = nullptr;
    TcCC* tcc = nullptr;  // expansion and projection on the tensor cores (split forms, many states)
    TcMT* tcmt = nullptr; // muffin-tin blocks on the tensor cores (split-BF16 form, many states)
    zf* d_mtg = nullptr;  // muffin-tin stacks [h_eff; o; p] (FP32 forms, many states)
    zd* d_mtw = nullptr;
    zd* d_mtv = nullptr;  // per (k, atom) the gathered right-hand block [Q; C_lo] (m x N_s)
    int mtw_stride = 0, mtv_stride = 0;
    GemmDesc* gd_mt1 = nullptr;
    size_t nblk = 0;
    zd *d_vtab = nullptr, *d_dvtab = nullptr, *d_vstep = nullptr;
    zf *d_vtab32 = nullptr, *d_vstep32 = nullptr;
    uint2* d_vsteps = nullptr;  // pre-split per-step table (tensor-core forms)
    double tc_st = 1.0;         // its fp16 scale
    double *d_occ = nullptr, *d_wk = nullptr, *d_lam = nullptr;
    DevState* d_st = nullptr;
    double* d_rec = nullptr;
    double *d_part_jmt = nullptr, *d_part_full = nullptr, *d_part_post = nullptr;
    double *d_part_fin = nullptr, *d_gdev = nullptr;
    int max_nback = 1, wmax = 1, nseg = 1, segw = BT, ntsel = 2, msegw = 64, nslot = 1, coop_grid = 0;
    int toep_global = 0;  // the direct sum's table window does not fit in shared memory: gather from L2
    int cheb_tile = 0;
    zd* d_part_t = nullptr;
    zd* d_part = nullptr;
    double *d_a = nullptr, *d_dvs = nullptr;
    int call_cap = 0;
    int* d_flag = nullptr;
    GemmDesc *gd_expand = nullptr, *gd_fwd = nullptr, *gd_proj = nullptr, *gd_g1 = nullptr,
             *gd_g2 = nullptr, *gd_evh = nullptr, *gd_evn = nullptr;
    GemmDesc *gd_dvw = nullptr, *gd_dvg = nullptr, *gd_dvi = nullptr, *gd_dvi32 = nullptr;
    GemmDesc *gd_dvw32 = nullptr, *gd_dvg32 = nullptr;  // the muffin-tin rebuild in FP32 (reduced-precision forms)
    zf* d_dh32 = nullptr;
    // muffin-tin part of the density feedback
    zd *d_mtn0 = nullptr, *d_mty = nullptr;
    double *d_mt_lnorm = nullptr, *d_mt_fn2 = nullptr;
    GemmDesc* gd_mty = nullptr;
    zd* d_part_dv = nullptr;
    int kc_dvi = 0;
    ToepDesc* td_dv = nullptr;
    zd** d_jac_mats = nullptr;
    double** d_jac_vals = nullptr;
    zd** d_jac_vecs = nullptr;
    int kc_fwd = 0, kc_proj = 0, kc_expand = 0;
    std::vector<double> eps_min, eps_max, pnorm, dvnorm;
    std::vector<std::vector<int>> h_glin;       // host copy of the table offsets of G per k
    TcPlan* tc = nullptr;                       // tensor-core operator (split-BF16 form)
    FftPlan* fft = nullptr;                     // FFT route of the interstitial convolution
    ToepDesc* td_op = nullptr;                  // per k {C, th}: the operator's convolution
    unsigned* d_tile_cnt = nullptr;             // row-tile counters of the fused split-K sums
    GemmDesc* gd_exp64 = nullptr;               // Hartree feedback, FP32 form: C in FP64 for the density
    ToepDesc* td_dens = nullptr;                // per k {C of the density, -}
    cudaStream_t side = nullptr;                // the FFT route's interstitial rows overlap the matching rows
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    double dtcr0 = 0;
    int nterms = 0, launches_per_step = 0;
    bool dv_set = false;
    cudaGraphExec_t gexec = nullptr;
    int g_key_nterms = -1, g_key_dv = -1, g_key_steps = -1;
    int rec_count = 0;
    long long steps_done = 0;
    double time = 0.0;
    double a_max_cur = -1.0, s_max_cur = -1.0;  // bounds the Chebyshev interval was built for
    double* h_stage = nullptr;                  // pinned staging of host samples
    int stage_cap = 0;
    cudaEvent_t stage_ev = nullptr;
    std::string err;
};

// ------------------------------------------------------------ helpers
#define CK(x)                                                                            \
    do {                                                                                 \
        cudaError_t e_ = (x);                                                            \
        if (e_ != cudaSuccess) {                                                         \
            set_err(ctx, std::string(#x) + ": " + cudaGetErrorString(e_));               \
            throw Fail{e_ == cudaErrorMemoryAllocation ? RTTDDFT_ERR_OOM : RTTDDFT_ERR_CUDA}; \
        }                                                                                \
    } while (0)
#define KCHECK() CK(cudaGetLastError())

static void set_err(rttddft_ctx* ctx, const std::string& s) {
    if (ctx) ctx->err = s;
    g_last_error = s;
}
[[noreturn]] static void fail(rttddft_ctx* ctx, int code, const std::string& s) {
    set_err(ctx, s);
    throw Fail{code};
}

template <typename T>
static T* dalloc(rttddft_ctx* ctx, size_t n) {
    if (n == 0) n = 1;
    void* p = nullptr;
    CK(cudaMalloc(&p, n * sizeof(T)));
    ctx->allocs.push_back(p);
    return (T*)p;
}
template <typename T>
static T* dupload(rttddft_ctx* ctx, const T* h, size_t n) {
    T* d = dalloc<T>(ctx, n);
    if (n) CK(cudaMemcpy(d, h, n * sizeof(T), cudaMemcpyHostToDevice));
    return d;
}
static void dfree(rttddft_ctx* ctx, void* p) {
    if (!p) return;
    auto it = std::find(ctx->allocs.begin(), ctx->allocs.end(), p);
    if (it != ctx->allocs.end()) ctx->allocs.erase(it);
    cudaFree(p);
}

static bool finite_all(const double* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// max |M - M^H| / max(1, max |M|) for a complex column-major m x m block
static double herm_dev(const double* m2, int m) {
    const cplx* M = (const cplx*)m2;
    double dev = 0.0, mx = 1.0;
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) {
            dev = std::max(dev, std::abs(M[i + (size_t)j * m] - std::conj(M[j + (size_t)i * m])));
            mx = std::max(mx, std::abs(M[i + (size_t)j * m]));
        }
    return dev / mx;
}

// Cholesky test for positive definiteness of a Hermitian block
static bool is_pd(const double* m2, int m) {
    const cplx* M = (const cplx*)m2;
    std::vector<cplx> L((size_t)m * m, 0.0);
    for (int j = 0; j < m; ++j) {
        double d = M[j + (size_t)j * m].real();
        for (int k = 0; k < j; ++k) d -= std::norm(L[j + (size_t)k * m]);
        if (!(d > 0.0)) return false;
        const double ljj = sqrt(d);
        L[j + (size_t)j * m] = ljj;
        for (int i = j + 1; i < m; ++i) {
            cplx s = M[i + (size_t)j * m];
            for (int k = 0; k < j; ++k) s -= L[i + (size_t)k * m] * std::conj(L[j + (size_t)k * m]);
            L[i + (size_t)j * m] = s / ljj;
        }
    }
    return true;
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static GemmDesc* upload_descs(rttddft_ctx* ctx, const std::vector<GemmDesc>& v) {
    return dupload(ctx, v.data(), v.size());
}

static StepArgs make_args(rttddft_ctx* ctx, int dv_on) {
    StepArgs a{};
    a.nk = ctx->nk;
    a.ns = ctx->ns;
    a.naux = ctx->naux;
    a.prop = ctx->opt.propagator;
    a.prec = ctx->opt.precision;
    a.reproject = ctx->opt.reproject;
    a.nterms = ctx->nterms;
    a.dv_on = dv_on;
    a.vt_center = ctx->vt_center;
    a.nvt = ctx->nvt;
    a.lrows = ctx->at.lrows;
    a.ma = ctx->at.ma;
    a.rec_cap = ctx->opt.max_record;
    a.dt = ctx->opt.dt;
    a.c = ctx->c;
    a.inv_c = 1.0 / ctx->c;
    a.half_inv_c2 = 0.5 / (ctx->c * ctx->c);
    a.omega = ctx->omega;
    a.kd = ctx->d_kd;
    a.occ = ctx->d_occ;
    a.wk = ctx->d_wk;
    a.h = ctx->d_h;
    a.o = ctx->d_o;
    a.p = ctx->d_p;
    a.h32 = ctx->d_h32;
    a.o32 = ctx->d_o32;
    a.p32 = ctx->d_p32;
    a.dh = dv_on ? ctx->d_dh : nullptr;
    a.vtab = ctx->d_vtab;
    a.vtab32 = ctx->d_vtab32;
    a.dvtab = ctx->d_dvtab;
    a.vstep = ctx->d_vstep;
    a.vstep32 = ctx->d_vstep32;
    a.vsteps = ctx->d_vsteps;
    a.a = ctx->d_a;
    a.dvs = (dv_on && !ctx->opt.hartree) ? ctx->d_dvs : nullptr;  // the density feedback runs with s = 1
    a.st = ctx->d_st;
    a.rec = ctx->d_rec;
    a.part_jmt = ctx->d_part_jmt;
    a.part_full = ctx->d_part_full;
    a.part_post = ctx->d_part_post;
    a.part_fin = ctx->d_part_fin;
    a.mt_u = (ctx->opt.hartree && ctx->d_mtn0) ? ctx->opt.hartree_mt_u : 0.0;
    a.mtn0 = ctx->d_mtn0;
    a.mty = ctx->d_mty;
    a.mt_lnorm = ctx->d_mt_lnorm;
    a.mt_fn2 = ctx->d_mt_fn2;
    a.dh32 = ctx->d_dh32;
    a.gdev = ctx->d_gdev;
    a.at = ctx->d_at;
    a.gd_proj = ctx->gd_proj;
    a.part_proj = ctx->d_part;
    a.kc_proj = ctx->kc_proj;
    a.max_nback = ctx->max_nback;
    a.wmax = ctx->wmax;
    a.nseg = ctx->nseg;
    a.segw = ctx->segw;
    a.maxng = ctx->maxng;
    a.msegw = ctx->msegw;
    a.nslot = ctx->nslot;
    a.part_t = ctx->d_part_t;
    a.flag = ctx->d_flag;
    a.coop_grid = ctx->coop_grid;
    a.cheb_tile = ctx->cheb_tile;
    a.tcback = (ctx->opt.precision >= RTTDDFT_PREC_BF16X3 && tc_has_back(ctx->tc)) ? 1 : 0;
    a.tc_fmt = tc_format(ctx->tc);
    a.tc_st = tc_table_scale(ctx->tc);
    a.at_n = ctx->at.n;
    a.at_maxm = ctx->maxm;
    a.ith = (ctx->opt.precision >= RTTDDFT_PREC_BF16X3 || ctx->fft || ctx->toep_global) ? 1 : 0;
    a.toep_global = ctx->toep_global;
    a.hartree = ctx->opt.hartree;
    a.mtg = ctx->d_mtg;
    a.mtw = ctx->d_mtw;
    a.mtv = ctx->d_mtv;
    a.mtv_stride = ctx->mtv_stride;
    a.mtw_stride = ctx->mtw_stride;
    return a;
}

static void build_mt_rebuild(rttddft_ctx* ctx);

static StepPlan make_plan(rttddft_ctx* ctx) {
    StepPlan p{};
    p.maxnb = ctx->maxnb;
    p.maxng = ctx->maxng;
    p.nterms = ctx->nterms;
    p.gd_expand = ctx->gd_expand;
    p.gd_fwd = ctx->gd_fwd;
    p.gd_proj = ctx->gd_proj;
    p.gd_g1 = ctx->gd_g1;
    p.gd_g2 = ctx->gd_g2;
    p.gd_evh = ctx->gd_evh;
    p.gd_evn = ctx->gd_evn;
    p.part = ctx->d_part;
    p.kc_fwd = ctx->kc_fwd;
    p.kc_proj = ctx->kc_proj;
    p.kc_expand = ctx->kc_expand;
    p.gd_dvw = ctx->gd_dvw;
    p.gd_dvg = ctx->gd_dvg;
    p.gd_dvi = ctx->gd_dvi;
    p.gd_dvi32 = ctx->gd_dvi32;
    p.gd_dvw32 = ctx->gd_dvw32;
    p.gd_dvg32 = ctx->gd_dvg32;
    p.part_dv = ctx->d_part_dv;
    p.kc_dvi = ctx->kc_dvi;
    p.td_dv = ctx->td_dv;
    p.n_dvw = ctx->nk * ctx->at.n;
    p.maxm = ctx->maxm;
    p.d_flag = ctx->d_flag;
    p.jac_mats = ctx->d_jac_mats;
    p.jac_vals = ctx->d_jac_vals;
    p.jac_vecs = ctx->d_jac_vecs;
    p.max_sweeps = ctx->opt.max_sweeps;
    p.tc = ctx->tc;
    p.tcc = ctx->tcc;
    p.tcmt = ctx->tcmt;
    p.fft = ctx->fft;
    p.td_op = ctx->td_op;
    p.tile_cnt = ctx->d_tile_cnt;
    p.side = ctx->side;
    p.ev_fork = ctx->ev_fork;
    p.ev_join = ctx->ev_join;
    p.gd_exp64 = ctx->gd_exp64;
    p.gd_mt1 = ctx->gd_mt1;
    p.gd_mty = ctx->gd_mty;
    p.td_dens = ctx->td_dens ? ctx->td_dens : ctx->td_op;
    {
        int F[3], fused = 0;
        fft_plan_info(ctx->fft, F, &fused);
        p.fft_launches = ctx->fft ? (fused ? 3 : 5) : 0;
    }
    return p;
}

// rows of C per block of the CN kernel for N right-hand columns
static int cn_rows(int N) { return N <= 2 ? 32 : (N <= 4 ? 16 : 8); }

// K-chunk of a split-K launch so that about two blocks per SM are busy
static int kchunk_for(int tiles_per_batch, int nbatch, int maxK) {
    const int target = 2 * 152;
    int splits = (target + tiles_per_batch * nbatch - 1) / (tiles_per_batch * nbatch);
    splits = std::max(1, std::min(splits, (maxK + 255) / 256));
    int kc = (maxK + splits - 1) / splits;
    kc = (kc + 127) / 128 * 128;
    return std::max(kc, 128);
}

// ------------------------------------------------------------ set-up pieces
// Local coordinates L = [A_alpha X_G ; X_lo(alpha)] stacked over atoms,
// lrows x ncol per k, for X given per k (nb x ncol, ld nb).
static void local_coords(rttddft_ctx* ctx, const std::vector<zd*>& X, const std::vector<zd*>& L,
                         int ncol) {
    const AtomTab& at = ctx->at;
    if (at.n == 0) return;
    std::vector<GemmDesc> v;
    std::vector<GemmDesc> cp;
    for (int k = 0; k < ctx->nk; ++k) {
        for (int a = 0; a < at.n; ++a) {
            GemmDesc g{};
            g.A = ctx->hkd[k].at + (size_t)at.aoff[a] * ctx->ng[k];  // columns of A^H
            g.B = X[k];
            g.C = L[k] + at.loff[a];
            g.M = at.na[a];
            g.K = ctx->ng[k];
            g.lda = ctx->ng[k];
            g.ldb = ctx->nb[k];
            g.ldc = at.lrows;
            v.push_back(g);
            // LO rows: L[loff + na + j] = X[ng + looff + j] as a product with the identity
            // is avoided: copy through a GEMM with K = 0 is not possible, so use a
            // strided copy descriptor (A = X rows, M = nlo)
            GemmDesc c{};
            c.B = X[k] + ctx->ng[k] + at.looff[a];
            c.C = L[k] + at.loff[a] + at.na[a];
            c.M = at.nlo[a];
            c.K = ncol;
            c.ldb = ctx->nb[k];
            c.ldc = at.lrows;
            cp.push_back(c);
        }
    }
    GemmDesc* d = upload_descs(ctx, v);
    int maxna = 0;
    for (int a = 0; a < at.n; ++a) maxna = std::max(maxna, at.na[a]);
    launch_gemm_cn(d, (int)v.size(), maxna, ctx->maxng, ncol, 0, nullptr, 0, false, nullptr, ctx->stream);
    KCHECK();
    GemmDesc* dc = upload_descs(ctx, cp);
    int maxlo = 0;
    for (int a = 0; a < at.n; ++a) maxlo = std::max(maxlo, at.nlo[a]);
    if (maxlo > 0) launch_copy_rows(dc, (int)cp.size(), maxlo, ncol, ctx->stream);
    KCHECK();
    CK(cudaStreamSynchronize(ctx->stream));
    dfree(ctx, d);
    dfree(ctx, dc);
}

// G[k] = X^H M X for M in {S (which=0), H0 (1), P_l (2 + l)}, ncol x ncol per k,
// from the local coordinates L of X and the plane-wave rows of X.
static void gram(rttddft_ctx* ctx, int which, const std::vector<zd*>& X, const std::vector<zd*>& L,
                 const std::vector<zd*>& G, int ncol, const zd* tab_override = nullptr,
                 const zd* blocks_override = nullptr) {
    const AtomTab& at = ctx->at;
    const int nk = ctx->nk;
    std::vector<zd*> W(nk), T(nk);
    for (int k = 0; k < nk; ++k) {
        W[k] = dalloc<zd>(ctx, (size_t)std::max(at.lrows, 1) * ncol);
        T[k] = dalloc<zd>(ctx, (size_t)ctx->ng[k] * ncol);
    }
    // muffin-tin part: W = blockdiag(M_alpha) L, G = L^H W
    if (at.n > 0) {
        std::vector<GemmDesc> v;
        for (int k = 0; k < nk; ++k)
            for (int a = 0; a < at.n; ++a) {
                GemmDesc g{};
                const zd* blk;
                if (blocks_override) blk = blocks_override + at.boff[a];
                else if (which == 0) blk = ctx->d_o + at.boff[a];
                else if (which == 1) blk = ctx->d_h + at.boff[a];
                else blk = ctx->d_p + 3 * at.boff[a] + (size_t)(which - 2) * at.m[a] * at.m[a];
                g.A = blk;
                g.B = L[k] + at.loff[a];
                g.C = W[k] + at.loff[a];
                g.M = at.m[a];
                g.K = at.m[a];
                g.lda = at.m[a];
                g.ldb = at.lrows;
                g.ldc = at.lrows;
                v.push_back(g);
            }
        GemmDesc* d = upload_descs(ctx, v);
        launch_gemm_nn(d, (int)v.size(), ctx->maxm, ctx->maxm, ncol, 0, nullptr, 0, false, nullptr,
                       ctx->stream);
        KCHECK();
        std::vector<GemmDesc> u;
        for (int k = 0; k < nk; ++k) {
            GemmDesc g{};
            g.A = L[k];
            g.B = W[k];
            g.C = G[k];
            g.M = ncol;
            g.K = at.lrows;
            g.lda = at.lrows;
            g.ldb = at.lrows;
            g.ldc = ncol;
            u.push_back(g);
        }
        GemmDesc* d2 = upload_descs(ctx, u);
        launch_gemm_cn(d2, nk, ncol, at.lrows, ncol, 0, nullptr, 0, false, nullptr, ctx->stream);
        KCHECK();
        CK(cudaStreamSynchronize(ctx->stream));
        dfree(ctx, d);
        dfree(ctx, d2);
    } else {
        for (int k = 0; k < nk; ++k) launch_zero(G[k], (size_t)ncol * ncol, ctx->stream);
    }
    // plane-wave part: T = (table * X_G) + d_G X_G, G += X_G^H T
    std::vector<ToepDesc> tdv(nk);
    for (int k = 0; k < nk; ++k) tdv[k] = ToepDesc{X[k], T[k], ctx->nb[k], ctx->ng[k]};
    ToepDesc* td = dupload(ctx, tdv.data(), tdv.size());
    const zd* tab = nullptr;
    int dmode = 0;
    if (which == 0) dmode = 5;
    else if (which == 1) {
        tab = ctx->d_vtab;
        dmode = 1;
    } else if (which >= 2 && which <= 4) dmode = which;
    else if (which == 9) tab = tab_override;  // potential change: table only
    launch_toeplitz(ctx->d_kd, td, nk, ctx->maxng, ncol, tab, ctx->vt_center, 0, dmode, nullptr,
                    ctx->stream);
    KCHECK();
    std::vector<GemmDesc> u;
    for (int k = 0; k < nk; ++k) {
        GemmDesc g{};
        g.A = X[k];
        g.B = T[k];
        g.C = G[k];
        g.M = ncol;
        g.K = ctx->ng[k];
        g.lda = ctx->nb[k];
        g.ldb = ctx->ng[k];
        g.ldc = ncol;
        u.push_back(g);
    }
    GemmDesc* d3 = upload_descs(ctx, u);
    int kc = kchunk_for((ncol + 7) / 8, nk, ctx->maxng);
    size_t pe = 0;
    for (int k = 0; k < nk; ++k) {
        u[k].part_off = pe;
        pe += (size_t)((ctx->ng[k] + kc - 1) / kc) * ncol * ncol;
    }
    CK(cudaMemcpy(d3, u.data(), u.size() * sizeof(GemmDesc), cudaMemcpyHostToDevice));
    zd* part = dalloc<zd>(ctx, pe);
    launch_gemm_cn(d3, nk, ncol, ctx->maxng, ncol, kc, part, 0, false, nullptr, ctx->stream);
    launch_split_reduce(d3, nk, ncol, ncol, kc, part, 1, ctx->stream);
    KCHECK();
    CK(cudaStreamSynchronize(ctx->stream));
    dfree(ctx, part);
    dfree(ctx, d3);
    dfree(ctx, td);
    for (int k = 0; k < nk; ++k) {
        dfree(ctx, W[k]);
        dfree(ctx, T[k]);
    }
}

// batched square GEMMs on per-k naux x naux matrices
static void sq_gemm(rttddft_ctx* ctx, bool conjA, const std::vector<zd*>& A, const std::vector<zd*>& B,
                    const std::vector<zd*>& C, int n) {
    std::vector<GemmDesc> v;
    for (int k = 0; k < ctx->nk; ++k) {
        GemmDesc g{};
        g.A = A[k];
        g.B = B[k];
        g.C = C[k];
        g.M = n;
        g.K = n;
        g.lda = n;
        g.ldb = n;
        g.ldc = n;
        v.push_back(g);
    }
    GemmDesc* d = upload_descs(ctx, v);
    if (conjA) launch_gemm_cn(d, ctx->nk, n, n, n, 0, nullptr, 0, false, nullptr, ctx->stream);
    else launch_gemm_nn(d, ctx->nk, n, n, n, 0, nullptr, 0, false, nullptr, ctx->stream);
    KCHECK();
    CK(cudaStreamSynchronize(ctx->stream));
    dfree(ctx, d);
}

static void jacobi(rttddft_ctx* ctx, const std::vector<zd*>& mats, const std::vector<double*>& vals,
                   const std::vector<zd*>& vecs, int n) {
    zd** dm = dupload(ctx, mats.data(), mats.size());
    double** dv = dupload(ctx, vals.data(), vals.size());
    zd** dx = dupload(ctx, vecs.data(), vecs.size());
    CK(cudaMemset(ctx->d_flag, 0, sizeof(int)));
    if (launch_jacobi(dm, dv, dx, (int)mats.size(), n, ctx->opt.max_sweeps, ctx->d_flag, ctx->stream))
        fail(ctx, RTTDDFT_ERR_UNSUPPORTED, "n_aux above the eigensolver limit (1024)");
    KCHECK();
    CK(cudaStreamSynchronize(ctx->stream));
    int flag = 0;
    CK(cudaMemcpy(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost));
    dfree(ctx, dm);
    dfree(ctx, dv);
    dfree(ctx, dx);
    if (flag) fail(ctx, RTTDDFT_ERR_TIMEOUT, "Jacobi eigensolver reached its sweep limit");
}


static void validate(const rttddft_system* s, const rttddft_options* o) {
    rttddft_ctx* ctx = nullptr;
    if (!s) fail(ctx, RTTDDFT_ERR_ARG, "system is NULL");
    if (s->n_k < 1) fail(ctx, RTTDDFT_ERR_ARG, "n_k < 1");
    if (s->n_atoms < 0 || s->n_atoms > RTD_MAX_ATOMS) fail(ctx, RTTDDFT_ERR_ARG, "n_atoms out of range [0, 64]");
    if (s->n_s < 1 || s->n_aux < s->n_s) fail(ctx, RTTDDFT_ERR_ARG, "need 1 <= n_s <= n_aux");
    if (s->n_aux > 1024) fail(ctx, RTTDDFT_ERR_UNSUPPORTED, "n_aux > 1024");
    if (!(s->omega > 0) || !(s->c_light > 0)) fail(ctx, RTTDDFT_ERR_ARG, "omega and c_light must be > 0");
    if (!s->occ || !s->wk || !s->n_g || !s->g_int || !s->gk || !s->vtab || !s->caux)
        fail(ctx, RTTDDFT_ERR_ARG, "NULL array in system");
    if (s->n_atoms > 0 && (!s->n_a || !s->n_lo || !s->amat || !s->h || !s->o || !s->p))
        fail(ctx, RTTDDFT_ERR_ARG, "NULL atom array in system");
    for (int i = 0; i < 3; ++i)
        if (s->vt_dim[i] < 1 || (s->vt_dim[i] & 1) == 0) fail(ctx, RTTDDFT_ERR_ARG, "vt_dim must be odd and >= 1");
    if (!o) fail(ctx, RTTDDFT_ERR_ARG, "options are NULL");
    if (!(o->dt > 0)) fail(ctx, RTTDDFT_ERR_ARG, "dt must be > 0");
    if (o->propagator < 0 || o->propagator > 2) fail(ctx, RTTDDFT_ERR_UNSUPPORTED, "unknown propagator");
    if (o->precision < 0 || o->precision > 3) fail(ctx, RTTDDFT_ERR_UNSUPPORTED, "unknown precision form");
    if (o->interstitial != RTTDDFT_INTERSTITIAL_TOEPLITZ && o->interstitial != RTTDDFT_INTERSTITIAL_FFT)
        fail(ctx, RTTDDFT_ERR_UNSUPPORTED, "unknown interstitial route");
    if (o->hartree != 0 && o->hartree != 1) fail(ctx, RTTDDFT_ERR_ARG, "hartree must be 0 or 1");
    if (o->hartree) {
        if (o->interstitial != RTTDDFT_INTERSTITIAL_FFT)
            fail(ctx, RTTDDFT_ERR_UNSUPPORTED, "the Hartree feedback needs the FFT interstitial route");
        if (!(o->hartree_bound > 0.0) || !std::isfinite(o->hartree_bound))
            fail(ctx, RTTDDFT_ERR_ARG, "hartree_bound must be positive");
        if (!std::isfinite(o->hartree_mt_u)) fail(ctx, RTTDDFT_ERR_NONFINITE, "hartree_mt_u not finite");
        double r2 = 0.0;
        for (int i = 0; i < 9; ++i) {
            if (!std::isfinite(s->recip[i])) fail(ctx, RTTDDFT_ERR_NONFINITE, "recip not finite");
            r2 += s->recip[i] * s->recip[i];
        }
        if (r2 == 0.0) fail(ctx, RTTDDFT_ERR_ARG, "the Hartree feedback needs the reciprocal vectors (recip)");
    }
    if (o->aux_mode < 0 || o->aux_mode > 1) fail(ctx, RTTDDFT_ERR_UNSUPPORTED, "unknown aux_mode");
    if (o->aux_mode == RTTDDFT_AUX_GIVEN && !s->eps) fail(ctx, RTTDDFT_ERR_ARG, "GIVEN mode needs eps");
    if (o->max_record < 1 || o->graph_steps < 0 || o->max_sweeps < 1) fail(ctx, RTTDDFT_ERR_ARG, "bad option value");
    if (!finite_all(s->occ, s->n_s) || !finite_all(s->wk, s->n_k)) fail(ctx, RTTDDFT_ERR_NONFINITE, "occ/wk not finite");
}

// ------------------------------------------------------------ ABI
extern "C" {

void rttddft_default_options(rttddft_options* opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->dt = 0.1;
    opt->propagator = RTTDDFT_PROP_CHEBYSHEV;
    opt->precision = RTTDDFT_PREC_FP64;
    opt->reproject = 0;
    opt->aux_mode = RTTDDFT_AUX_RITZ;
    opt->max_record = 4096;
    opt->graph_steps = 1;
    opt->cheb_tol = 1e-16;
    opt->ortho_tol = 1e-10;
    opt->max_sweeps = 30;
    opt->a_max = 0.0;
    opt->s_max = 0.0;
    opt->interstitial = RTTDDFT_INTERSTITIAL_TOEPLITZ;
    opt->hartree = 0;
    opt->hartree_bound = 0.1;
    opt->hartree_mt_u = 0.0;
}

const char* rttddft_version(void) { return "rttddft-gb300 0.1 (sm_103a)"; }

const char* rttddft_last_error(const rttddft_ctx* ctx) {
    if (ctx) return ctx->err.c_str();
    return g_last_error.c_str();
}

void rttddft_destroy(rttddft_ctx* ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    tc_plan_destroy(ctx->tc);
    tc_cc_destroy(ctx->tcc);
    tc_mt_destroy(ctx->tcmt);
    fft_plan_destroy(ctx->fft);
    for (void* p : ctx->allocs) cudaFree(p);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    if (ctx->stage_ev) cudaEventDestroy(ctx->stage_ev);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

int rttddft_setup(const rttddft_system* s, const rttddft_options* opt_in, void* cuda_stream,
                  rttddft_ctx** out) {
    rttddft_ctx* ctx = nullptr;
    if (!out) {
        g_last_error = "out is NULL";
        return RTTDDFT_ERR_ARG;
    }
    *out = nullptr;
    rttddft_options dflt;
    rttddft_default_options(&dflt);
    const rttddft_options* o = opt_in ? opt_in : &dflt;
    try {
        validate(s, o);
        ctx = new rttddft_ctx();
        ctx->opt = *o;
        ctx->nk = s->n_k;
        ctx->natoms = s->n_atoms;
        ctx->ns = s->n_s;
        ctx->naux = s->n_aux;
        ctx->omega = s->omega;
        ctx->c = s->c_light;
        const int nk = ctx->nk, ns = ctx->ns, naux = ctx->naux;
        // ---- atoms
        AtomTab& at = ctx->at;
        at.n = s->n_atoms;
        size_t boff = 0;
        int aoff = 0, looff = 0, loff = 0;
        for (int a = 0; a < at.n; ++a) {
            if (s->n_a[a] < 0 || s->n_lo[a] < 0 || s->n_a[a] + s->n_lo[a] < 1)
                fail(ctx, RTTDDFT_ERR_ARG, "atom with no rows");
            at.na[a] = s->n_a[a];
            at.nlo[a] = s->n_lo[a];
            at.m[a] = at.na[a] + at.nlo[a];
            at.aoff[a] = aoff;
            at.looff[a] = looff;
            at.loff[a] = loff;
            at.boff[a] = boff;
            aoff += at.na[a];
            looff += at.nlo[a];
            loff += at.m[a];
            boff += (size_t)at.m[a] * at.m[a];
            ctx->maxm = std::max(ctx->maxm, at.m[a]);
        }
        at.ma = aoff;
        at.nlo_tot = looff;
        at.lrows = loff;
        const size_t nblk = boff;
        // ---- host validation of the blocks and the table
        if (at.n > 0) {
            if (!finite_all(s->h, 2 * nblk) || !finite_all(s->o, 2 * nblk) || !finite_all(s->p, 6 * nblk))
                fail(ctx, RTTDDFT_ERR_NONFINITE, "muffin-tin block not finite");
            for (int a = 0; a < at.n; ++a) {
                const int m = at.m[a];
                const double* hb = s->h + 2 * at.boff[a];
                const double* ob = s->o + 2 * at.boff[a];
                if (herm_dev(hb, m) > 1e-12 || herm_dev(ob, m) > 1e-12)
                    fail(ctx, RTTDDFT_ERR_NOT_HERMITIAN, "h or o block of atom " + std::to_string(a) + " not Hermitian");
                for (int l = 0; l < 3; ++l)
                    if (herm_dev(s->p + 2 * (3 * at.boff[a] + (size_t)l * m * m), m) > 1e-12)
                        fail(ctx, RTTDDFT_ERR_NOT_HERMITIAN, "p block of atom " + std::to_string(a) + " not Hermitian");
                if (!is_pd(ob, m)) fail(ctx, RTTDDFT_ERR_NOT_PD, "o block of atom " + std::to_string(a) + " not positive definite");
            }
        }
        for (int i = 0; i < 3; ++i) ctx->vt_dim[i] = s->vt_dim[i];
        const int d0 = s->vt_dim[0], d1 = s->vt_dim[1], d2 = s->vt_dim[2];
        ctx->nvt = d0 * d1 * d2;
        const int e0 = (d0 - 1) / 2, e1 = (d1 - 1) / 2, e2 = (d2 - 1) / 2;
        ctx->vt_center = (e0 * d1 + e1) * d2 + e2;
        if (!finite_all(s->vtab, 2 * (size_t)ctx->nvt)) fail(ctx, RTTDDFT_ERR_NONFINITE, "vtab not finite");
        {
            const cplx* V = (const cplx*)s->vtab;
            double dev = 0.0, mx = 1e-300;
            for (int i = 0; i < ctx->nvt; ++i) mx = std::max(mx, std::abs(V[i]));
            for (int i = 0; i < ctx->nvt; ++i) dev = std::max(dev, std::abs(V[i] - std::conj(V[ctx->nvt - 1 - i])));
            if (dev > 1e-12 * mx) fail(ctx, RTTDDFT_ERR_NOT_HERMITIAN, "vtab not Hermitian in g");
        }
        // ---- k-points
        ctx->ng.resize(nk);
        ctx->nb.resize(nk);
        size_t goff = 0, coff = 0, aoffk = 0;
        std::vector<size_t> g_off(nk), c_off(nk), a_off(nk);
        for (int k = 0; k < nk; ++k) {
            const int ng = s->n_g[k];
            if (ng < 1) fail(ctx, RTTDDFT_ERR_ARG, "n_g < 1");
            int mn[3] = {1 << 30, 1 << 30, 1 << 30}, mx[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
            for (int g = 0; g < ng; ++g) {
                const int* t = s->g_int + 3 * (goff + g);
                for (int i = 0; i < 3; ++i) {
                    mn[i] = std::min(mn[i], t[i]);
                    mx[i] = std::max(mx[i], t[i]);
                }
            }
            if (mx[0] - mn[0] > e0 || mx[1] - mn[1] > e1 || mx[2] - mn[2] > e2)
                fail(ctx, RTTDDFT_ERR_ARG, "vtab box does not cover the G - G' differences");
            ctx->ng[k] = ng;
            ctx->nb[k] = ng + at.nlo_tot;
            if (naux > ctx->nb[k]) fail(ctx, RTTDDFT_ERR_ARG, "n_aux > N_basis of a k-point");
            ctx->maxng = std::max(ctx->maxng, ng);
            ctx->maxnb = std::max(ctx->maxnb, ctx->nb[k]);
            g_off[k] = goff;
            c_off[k] = coff;
            a_off[k] = aoffk;
            goff += ng;
            coff += (size_t)ctx->nb[k] * naux;
            aoffk += (size_t)at.ma * ng;
        }
        if (!finite_all(s->gk, 3 * goff) || !finite_all(s->caux, 2 * coff) ||
            (at.n > 0 && !finite_all(s->amat, 2 * aoffk)))
            fail(ctx, RTTDDFT_ERR_NONFINITE, "gk, caux or amat not finite");
        if (s->eps && o->aux_mode == RTTDDFT_AUX_GIVEN && !finite_all(s->eps, (size_t)nk * naux))
            fail(ctx, RTTDDFT_ERR_NONFINITE, "eps not finite");
        if (s->c0) {
            size_t n0 = 0;
            for (int k = 0; k < nk; ++k) n0 += (size_t)ctx->nb[k] * ns;
            if (!finite_all(s->c0, 2 * n0)) fail(ctx, RTTDDFT_ERR_NONFINITE, "c0 not finite");
        }
        // ---- device state (all host checks are done)
        CK(cudaGetDevice(&ctx->device));
        if (cuda_stream) {
            ctx->stream = (cudaStream_t)cuda_stream;
        } else {
            CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
            ctx->own_stream = true;
        }
        ctx->d_occ = dupload(ctx, s->occ, ns);
        ctx->d_wk = dupload(ctx, s->wk, nk);
        if (at.n > 0) {
            ctx->nblk = nblk;
            ctx->d_h = dupload(ctx, (const zd*)s->h, nblk);
            ctx->d_o = dupload(ctx, (const zd*)s->o, nblk);
            ctx->d_p = dupload(ctx, (const zd*)s->p, 3 * nblk);
        }
        ctx->d_vtab = dupload(ctx, (const zd*)s->vtab, ctx->nvt);
        ctx->d_at = dupload(ctx, &at, 1);
        ctx->d_st = dalloc<DevState>(ctx, 1);
        CK(cudaMemset(ctx->d_st, 0, sizeof(DevState)));
        ctx->d_flag = dalloc<int>(ctx, 1);
        ctx->d_rec = dalloc<double>(ctx, (size_t)o->max_record * RTD_REC_STRIDE);
        ctx->d_lam = dalloc<double>(ctx, LAM_N * (size_t)nk);
        ctx->max_nback = (ctx->maxng + BKB - 1) / BKB;
        {
            // split the G' sum of the interstitial term so that ~4 blocks per SM work
            const int tiles = (ctx->maxng + BT - 1) / BT;
            int nseg = (4 * 152 + tiles * nk - 1) / (tiles * nk);
            nseg = std::max(1, std::min(nseg, tiles));
            ctx->segw = ((tiles + nseg - 1) / nseg) * BT;
            ctx->nseg = (ctx->maxng + ctx->segw - 1) / ctx->segw;
            ctx->ntsel = ns <= 2 ? 2 : (ns <= 4 ? 4 : 8);
            ctx->msegw = 64;
            ctx->nslot = ctx->nseg + (at.ma + ctx->msegw - 1) / ctx->msegw;
            ctx->d_part_t = dalloc<zd>(ctx, (size_t)nk * ctx->nslot * 2 * ctx->ntsel * ctx->maxng);
        }
        ctx->d_part_jmt = dalloc<double>(ctx, (size_t)nk * std::max(at.lrows, 1) * 5);
        // one counter per 8-row tile and k-point (the smallest row tile of the FP32 kernels)
        ctx->d_tile_cnt = dalloc<unsigned>(ctx, (size_t)nk * ((std::max(at.ma, 1) + 7) / 8));
        CK(cudaMemset(ctx->d_tile_cnt, 0, sizeof(unsigned) * nk * ((std::max(at.ma, 1) + 7) / 8)));
        ctx->d_part_full = dalloc<double>(ctx, (size_t)nk * ctx->max_nback * 5);
        ctx->d_part_post = dalloc<double>(ctx, (size_t)nk * naux * POST_STRIDE);
        ctx->d_part_fin = dalloc<double>(ctx, (size_t)nk * FIN_CH * FIN_STRIDE);
        ctx->d_gdev = dalloc<double>(ctx, (size_t)nk * ns);
        CK(cudaMemset(ctx->d_part_jmt, 0, sizeof(double) * nk * std::max(at.lrows, 1) * 5));
        CK(cudaMemset(ctx->d_part_post, 0, sizeof(double) * nk * naux * POST_STRIDE));
        ctx->call_cap = 1024;
        ctx->d_a = dalloc<double>(ctx, 3 * (size_t)ctx->call_cap);
        ctx->d_dvs = dalloc<double>(ctx, (size_t)ctx->call_cap);
        // ---- per-k buffers
        ctx->hkd.resize(nk);
        const size_t nn = (size_t)naux * naux;
        for (int k = 0; k < nk; ++k) {
            KDev& K = ctx->hkd[k];
            K.ng = ctx->ng[k];
            K.nb = ctx->nb[k];
            K.caux = dupload(ctx, (const zd*)s->caux + c_off[k], (size_t)K.nb * naux);
            if (at.n > 0) {
                // matching coefficients are kept as A^H (N_G x M_A): both the forward
                // product A C_G and the back-projection A^H Z then read coalesced
                zd* tmp = dupload(ctx, (const zd*)s->amat + a_off[k], (size_t)at.ma * K.ng);
                K.at = dalloc<zd>(ctx, (size_t)at.ma * K.ng);
                launch_conj_transpose(tmp, K.at, at.ma, K.ng, ctx->stream);
                KCHECK();
                CK(cudaStreamSynchronize(ctx->stream));
                dfree(ctx, tmp);
            } else {
                K.at = nullptr;
            }
            std::vector<int> gl(K.ng);
            for (int g = 0; g < K.ng; ++g) {
                const int* t = s->g_int + 3 * (g_off[k] + g);
                gl[g] = (t[0] * d1 + t[1]) * d2 + t[2];
            }
            K.glin = dupload(ctx, gl.data(), gl.size());
            ctx->h_glin.push_back(gl);
            K.gk = dupload(ctx, s->gk + 3 * g_off[k], 3 * (size_t)K.ng);
            K.eps = dalloc<double>(ctx, naux);
            K.psub = dalloc<zd>(ctx, 3 * nn);
            K.lloc = dalloc<zd>(ctx, (size_t)std::max(at.lrows, 1) * naux);
            K.theta = dalloc<zd>(ctx, (size_t)naux * ns);
            K.theta_t = dalloc<zd>(ctx, (size_t)naux * ns);
            K.ring = dalloc<zd>(ctx, 3 * (size_t)naux * ns);
            K.acc = dalloc<zd>(ctx, (size_t)naux * ns);
            K.hsub = dalloc<zd>(ctx, nn);
            K.C = dalloc<zd>(ctx, (size_t)K.nb * ns);
            K.Y = dalloc<zd>(ctx, (size_t)K.nb * 2 * ns);
            K.Q = dalloc<zd>(ctx, (size_t)std::max(at.ma, 1) * ns);
            K.Z = dalloc<zd>(ctx, (size_t)std::max(at.ma, 1) * 2 * ns);
            const bool tcf = o->precision >= RTTDDFT_PREC_BF16X3;
            const bool fftr = o->interstitial == RTTDDFT_INTERSTITIAL_FFT;
            K.th = (tcf || fftr) ? dalloc<zd>(ctx, (size_t)K.ng * ns) : nullptr;
            K.tb = (tcf && at.ma > 0) ? dalloc<zd>(ctx, (size_t)K.ng * 2 * ns) : nullptr;
            K.gram = dalloc<zd>(ctx, 2 * (size_t)ns * ns);
            K.evec = dalloc<zd>(ctx, nn);
            K.eval = dalloc<double>(ctx, naux);
            K.wtmp = dalloc<zd>(ctx, (size_t)naux * ns);
            K.coef = dalloc<zd>(ctx, RTD_MAX_TERMS);
            K.lam = ctx->d_lam + LAM_N * k;
        }
        ctx->d_kd = dupload(ctx, ctx->hkd.data(), nk);
        // largest table window of a (row tile, column tile) pair of the back kernel
        {
            int wm = 1;
            size_t goff2 = 0;
            for (int k = 0; k < nk; ++k) {
                const int ng = ctx->ng[k];
                int rmax = 0;
                for (int t0 = 0; t0 < ng; t0 += BT) {
                    const int* a0 = s->g_int + 3 * (goff2 + t0);
                    const int* a1 = s->g_int + 3 * (goff2 + std::min(t0 + BT, ng) - 1);
                    const int l0 = (a0[0] * d1 + a0[1]) * d2 + a0[2];
                    const int l1 = (a1[0] * d1 + a1[1]) * d2 + a1[2];
                    rmax = std::max(rmax, l1 - l0);
                }
                wm = std::max(wm, 2 * rmax + 1);
                goff2 += ng;
            }
            ctx->wmax = wm;
            // the slot kernel stages the window next to a BT x 8 tile of the right operand;
            // a window beyond shared memory (G sets whose 128-row tiles span several planes
            // of the table) makes the direct sum gather the table through L1/L2 instead
            int dev = 0, smax = 0;
            CK(cudaGetDevice(&dev));
            CK(cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
            const size_t cb = o->precision == RTTDDFT_PREC_FP64 ? sizeof(zd) : sizeof(zf);  // the form's table entries
            const size_t need = (size_t)BT * 8 * cb + BT * sizeof(int) + (size_t)wm * cb;
            // RTTDDFT_TOEP_GATHER=1 in the environment takes the gather path at any size (tests)
            const char* force = getenv("RTTDDFT_TOEP_GATHER");
            if (need + 1024 > (size_t)smax || (force && force[0] == '1')) {
                ctx->toep_global = 1;
                ctx->wmax = 1;
                for (int k = 0; k < nk; ++k)
                    if (!ctx->hkd[k].th) ctx->hkd[k].th = dalloc<zd>(ctx, (size_t)ctx->hkd[k].ng * ns);
                CK(cudaMemcpy(ctx->d_kd, ctx->hkd.data(), nk * sizeof(KDev), cudaMemcpyHostToDevice));
            }
        }
        // ---- auxiliary basis
        std::vector<zd*> X(nk), L(nk), G1(nk), G2(nk), V1(nk), V2(nk), T1(nk), T2(nk), NEW(nk);
        std::vector<double*> E1(nk), E2(nk);
        for (int k = 0; k < nk; ++k) {
            X[k] = ctx->hkd[k].caux;
            L[k] = ctx->hkd[k].lloc;
            G1[k] = dalloc<zd>(ctx, nn);
            G2[k] = dalloc<zd>(ctx, nn);
            V1[k] = dalloc<zd>(ctx, nn);
            V2[k] = dalloc<zd>(ctx, nn);
            T1[k] = dalloc<zd>(ctx, nn);
            T2[k] = dalloc<zd>(ctx, nn);
            E1[k] = dalloc<double>(ctx, naux);
            E2[k] = ctx->hkd[k].eps;
        }
        local_coords(ctx, X, L, naux);
        gram(ctx, 0, X, L, G1, naux);  // X^H S X
        if (o->aux_mode == RTTDDFT_AUX_RITZ) {
            gram(ctx, 1, X, L, G2, naux);  // X^H H0 X
            // canonical S-orthonormalisation: X^H S X = W diag(lam) W^H, T1 = W lam^{-1/2}
            jacobi(ctx, G1, E1, V1, naux);
            for (int k = 0; k < nk; ++k) {
                std::vector<double> ev(naux);
                CK(cudaMemcpy(ev.data(), E1[k], naux * sizeof(double), cudaMemcpyDeviceToHost));
                if (!(ev[0] > 1e-12 * ev[naux - 1]))
                    fail(ctx, RTTDDFT_ERR_NOT_PD, "trial vectors are (numerically) linearly dependent in the S metric");
            }
            {
                zd** dm = dupload(ctx, V1.data(), nk);
                double** dv = dupload(ctx, E1.data(), nk);
                launch_scale_cols(dm, dv, nk, naux, 0, ctx->stream);
                KCHECK();
                CK(cudaStreamSynchronize(ctx->stream));
                dfree(ctx, dm);
                dfree(ctx, dv);
            }
            sq_gemm(ctx, false, G2, V1, T1, naux);  // X^H H0 X T1
            sq_gemm(ctx, true, V1, T1, T2, naux);   // T1^H X^H H0 X T1
            jacobi(ctx, T2, E2, V2, naux);           // Ritz values (ascending) and vectors
            sq_gemm(ctx, false, V1, V2, T1, naux);  // coefficients of the Ritz vectors in X
            // CC = X T  (new buffer, then swap)
            std::vector<GemmDesc> v;
            for (int k = 0; k < nk; ++k) {
                NEW[k] = dalloc<zd>(ctx, (size_t)ctx->nb[k] * naux);
                GemmDesc g{};
                g.A = X[k];
                g.B = T1[k];
                g.C = NEW[k];
                g.M = ctx->nb[k];
                g.K = naux;
                g.lda = ctx->nb[k];
                g.ldb = naux;
                g.ldc = ctx->nb[k];
                v.push_back(g);
            }
            GemmDesc* d = upload_descs(ctx, v);
            launch_gemm_nn(d, nk, ctx->maxnb, naux, naux, 0, nullptr, 0, false, nullptr, ctx->stream);
            KCHECK();
            CK(cudaStreamSynchronize(ctx->stream));
            dfree(ctx, d);
            for (int k = 0; k < nk; ++k) {
                dfree(ctx, ctx->hkd[k].caux);
                ctx->hkd[k].caux = NEW[k];
                X[k] = NEW[k];
            }
            CK(cudaMemcpy(ctx->d_kd, ctx->hkd.data(), nk * sizeof(KDev), cudaMemcpyHostToDevice));
            launch_phase_fix(ctx->d_kd, nk, naux, nullptr, nullptr, 0, ctx->stream);
            KCHECK();
            CK(cudaStreamSynchronize(ctx->stream));
            local_coords(ctx, X, L, naux);
        } else {
            for (int k = 0; k < nk; ++k) {
                std::vector<cplx> g(nn);
                CK(cudaMemcpy(g.data(), G1[k], nn * sizeof(zd), cudaMemcpyDeviceToHost));
                double dev = 0.0;
                for (int j = 0; j < naux; ++j)
                    for (int i = 0; i < naux; ++i)
                        dev = std::max(dev, std::abs(g[i + (size_t)j * naux] - (i == j ? 1.0 : 0.0)));
                if (dev > o->ortho_tol)
                    fail(ctx, RTTDDFT_ERR_NOT_ORTHONORMAL, "given CC(0) is not S-orthonormal (max dev " + std::to_string(dev) + ")");
                CK(cudaMemcpy(E2[k], s->eps + (size_t)k * naux, naux * sizeof(double), cudaMemcpyHostToDevice));
            }
        }
        // ---- projected momentum PP_l = CC^H P_l CC (Eq. auxiliary_hamiltonian_with_parts)
        for (int l = 0; l < 3; ++l) {
            std::vector<zd*> P(nk);
            for (int k = 0; k < nk; ++k) P[k] = ctx->hkd[k].psub + (size_t)l * nn;
            gram(ctx, 2 + l, X, L, P, naux);
        }
        ctx->eps_min.resize(nk);
        ctx->eps_max.resize(nk);
        ctx->pnorm.assign(3 * nk, 0.0);
        ctx->dvnorm.assign(nk, 0.0);
        ctx->dtcr0 = 1e300;
        for (int k = 0; k < nk; ++k) {
            std::vector<double> ev(naux);
            CK(cudaMemcpy(ev.data(), E2[k], naux * sizeof(double), cudaMemcpyDeviceToHost));
            ctx->eps_min[k] = *std::min_element(ev.begin(), ev.end());
            ctx->eps_max[k] = *std::max_element(ev.begin(), ev.end());
            if (ctx->eps_max[k] > ctx->eps_min[k])
                ctx->dtcr0 = std::min(ctx->dtcr0, 0.2 / (ctx->eps_max[k] - ctx->eps_min[k]));
            std::vector<double> pp(2 * 3 * nn);
            CK(cudaMemcpy(pp.data(), ctx->hkd[k].psub, 3 * nn * sizeof(zd), cudaMemcpyDeviceToHost));
            for (int l = 0; l < 3; ++l) {
                double f = 0.0;
                for (size_t e = 0; e < 2 * nn; ++e) f += pp[2 * l * nn + e] * pp[2 * l * nn + e];
                ctx->pnorm[3 * k + l] = sqrt(f);
            }
        }
        for (int k = 0; k < nk; ++k) {
            dfree(ctx, G1[k]);
            dfree(ctx, G2[k]);
            dfree(ctx, V1[k]);
            dfree(ctx, V2[k]);
            dfree(ctx, T1[k]);
            dfree(ctx, T2[k]);
            dfree(ctx, E1[k]);
        }
        // ---- FP32 copies for the FP32 and split-BF16 forms
        if (o->precision != RTTDDFT_PREC_FP64) {
            for (int k = 0; k < nk; ++k) {
                KDev& K = ctx->hkd[k];
                K.caux32 = dalloc<zf>(ctx, (size_t)K.nb * naux);
                launch_convert_f32(K.caux, K.caux32, (size_t)K.nb * naux, ctx->stream);
                if (at.n > 0) {
                    K.at32 = dalloc<zf>(ctx, (size_t)at.ma * K.ng);
                    launch_convert_f32(K.at, K.at32, (size_t)at.ma * K.ng, ctx->stream);
                }
            }
            ctx->d_vtab32 = dalloc<zf>(ctx, ctx->nvt);
            launch_convert_f32(ctx->d_vtab, ctx->d_vtab32, ctx->nvt, ctx->stream);
            if (ctx->nblk > 0) {
                ctx->d_h32 = dalloc<zf>(ctx, ctx->nblk);
                ctx->d_o32 = dalloc<zf>(ctx, ctx->nblk);
                ctx->d_p32 = dalloc<zf>(ctx, 3 * ctx->nblk);
                launch_convert_f32(ctx->d_h, ctx->d_h32, ctx->nblk, ctx->stream);
                launch_convert_f32(ctx->d_o, ctx->d_o32, ctx->nblk, ctx->stream);
                launch_convert_f32(ctx->d_p, ctx->d_p32, 3 * ctx->nblk, ctx->stream);
            }
            KCHECK();
            CK(cudaStreamSynchronize(ctx->stream));
        }
        // ---- tensor-core operands of the split-BF16 and split-FP16 forms
        if (o->precision >= RTTDDFT_PREC_BF16X3) {
            std::vector<int> ngv(nk);
            std::vector<const int*> glp(nk);
            std::vector<const zd*> atp(nk);
            for (int k = 0; k < nk; ++k) {
                ngv[k] = ctx->hkd[k].ng;
                glp[k] = ctx->h_glin[k].data();
                atp[k] = ctx->hkd[k].at;
            }
            // fp16 operand scales: the largest |A| and |V~| to 2^14 (powers of two)
            double amax = 0.0, vmax = 0.0;
            if (at.n > 0) {
                size_t na = 0;
                for (int k = 0; k < nk; ++k) na += (size_t)at.ma * ctx->hkd[k].ng;
                for (size_t i = 0; i < 2 * na; ++i) amax = std::max(amax, std::fabs(s->amat[i]));
            }
            for (int i = 0; i < 2 * ctx->nvt; ++i) vmax = std::max(vmax, std::fabs(s->vtab[i]));
            auto pow2_scale = [](double m) { return m > 0.0 ? std::ldexp(1.0, 14 - (int)std::ceil(std::log2(m))) : 1.0; };
            // the per-step table V~ + s dV~ keeps a factor 4 of headroom
            ctx->tc_st = pow2_scale(vmax) * 0.25;
            std::string why;
            const int fmt = (o->precision == RTTDDFT_PREC_BF16X3) ? 1 : 0;
            const int e = tc_plan_create(&ctx->tc, nk, ns, at.ma, ngv.data(), glp.data(), atp.data(),
                                         ctx->d_vtab, ctx->nvt, ctx->vt_center, ctx->d_kd, fmt, pow2_scale(amax),
                                         ctx->tc_st, ctx->stream, &why);
            if (e) fail(ctx, e, std::string(fmt ? "split-BF16" : "split-FP16") + " form: " + why);
        }
        // ---- FFT route of the interstitial convolution
        if (o->interstitial == RTTDDFT_INTERSTITIAL_FFT) {
            std::vector<int> ngv(nk);
            std::vector<const int*> gp(nk);
            std::vector<ToepDesc> td(nk);
            for (int k = 0; k < nk; ++k) {
                const KDev& K = ctx->hkd[k];
                ngv[k] = K.ng;
                gp[k] = s->g_int + 3 * g_off[k];
                td[k] = ToepDesc{K.C, K.th, K.nb, K.ng};
            }
            std::string why;
            const int e = fft_plan_create(&ctx->fft, nk, ngv.data(), gp.data(), ctx->vt_dim, ctx->d_vtab, ns,
                                          o->precision == RTTDDFT_PREC_FP64 ? 0 : 1, ctx->stream, &why);
            if (e) fail(ctx, e, why);
            ctx->td_op = dupload(ctx, td.data(), td.size());
            if (fft_tune(ctx->fft, ctx->td_op, ns, ctx->stream)) fail(ctx, RTTDDFT_ERR_CUDA, "FFT route: set-up timing failed");
            CK(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
            KCHECK();
            CK(cudaStreamSynchronize(ctx->stream));
        }
        if (!ctx->td_op) {
            // the operator's interstitial source and destination per k: {C, th}
            std::vector<ToepDesc> td(nk);
            for (int k = 0; k < nk; ++k) td[k] = ToepDesc{ctx->hkd[k].C, ctx->hkd[k].th, ctx->hkd[k].nb, ctx->hkd[k].ng};
            ctx->td_op = dupload(ctx, td.data(), td.size());
        }
        CK(cudaMemcpy(ctx->d_kd, ctx->hkd.data(), nk * sizeof(KDev), cudaMemcpyHostToDevice));
        // ---- step descriptors
        const bool f32 = o->precision != RTTDDFT_PREC_FP64;
        std::vector<GemmDesc> ex, fw, pj, g1, g2, eh, en;
        ctx->kc_fwd = kchunk_for((at.ma + cn_rows(ns) - 1) / cn_rows(ns), nk, ctx->maxng);
        ctx->kc_proj = kchunk_for((naux + cn_rows(ns) - 1) / cn_rows(ns), nk, ctx->maxnb);
        if (f32) {
            // the FP32 streaming kernels take K slices of at most 256
            ctx->kc_fwd = std::min(ctx->kc_fwd, 256);
            ctx->kc_proj = std::min(ctx->kc_proj, 256);
        }
        // the FP32 64 x 64 tiled kernel (many states): split K only as far as
        // about four blocks per SM need, in slices of a multiple of 16
        auto zt_kc = [&](int M, int K) {
            const int tiles = ((M + 63) / 64) * ((ns + 63) / 64) * nk;
            const int splits = std::max(1, std::min((K + 255) / 256, (4 * 152 + tiles - 1) / tiles));
            return splits == 1 ? 0 : ((K + splits - 1) / splits + 15) / 16 * 16;
        };
        if (f32 && ns >= ZT_MIN_N) {
            const int kf = zt_kc(at.ma, ctx->maxng), kp = zt_kc(naux, ctx->maxnb);
            ctx->kc_fwd = kf > 0 ? kf : ctx->maxng;
            ctx->kc_proj = kp > 0 ? kp : ctx->maxnb;
        }
        if (o->precision >= RTTDDFT_PREC_BF16X3 && ns >= ZT_MIN_N && 2 * ns <= 128) {
            // split forms, many states: C = CC theta and CC^H (S C) on the tensor cores;
            // the projection's partials arrive as one slice per k-point
            std::vector<const zd*> cp(nk);
            std::vector<int> nbv(nk);
            for (int k = 0; k < nk; ++k) {
                cp[k] = ctx->hkd[k].caux;
                nbv[k] = ctx->hkd[k].nb;
            }
            std::string why;
            const int e = tc_cc_create(&ctx->tcc, nk, naux, ns, nbv.data(), cp.data(), ctx->d_flag, ctx->stream, &why);
            if (e) fail(ctx, e, why);
            ctx->kc_proj = ctx->maxnb;
        }
        {
            // expand: rows are many, K = n_aux is short; split K only in FP64 where the
            // DFMA pipe of every SM is needed
            const int tiles = (ctx->maxnb + 63) / 64;
            ctx->kc_expand = 0;
            if (f32 && ns >= ZT_MIN_N) {
                ctx->kc_expand = zt_kc(ctx->maxnb, naux);
            } else if (f32) {
                // FP32 streaming kernel: K slices of at most 256; split only while the
                // row tiles alone leave most SMs idle (a split costs a reduction launch)
                int splits = (naux + 255) / 256;
                if (tiles * nk < 64) splits = std::max(splits, (2 * 152 + tiles * nk - 1) / (tiles * nk));
                splits = std::min(splits, std::max(1, naux / 32));
                if (splits > 1) ctx->kc_expand = (naux + splits - 1) / splits;
            } else if (tiles * nk < 2 * 152 && naux >= 128) {
                int splits = std::min((2 * 152 + tiles * nk - 1) / (tiles * nk), naux / 64);
                if (splits > 1) ctx->kc_expand = ((naux + splits - 1) / splits + 63) / 64 * 64;
            }
        }
        size_t pf = 0, pp = 0, pe = 0;
        for (int k = 0; k < nk; ++k) {
            KDev& K = ctx->hkd[k];
            GemmDesc g{};
            g.A = f32 ? (const void*)K.caux32 : (const void*)K.caux;
            g.B = K.theta;
            g.C = K.C;
            g.M = K.nb;
            g.K = naux;
            g.lda = K.nb;
            g.ldb = naux;
            g.ldc = K.nb;
            g.part_off = pe;
            if (ctx->kc_expand > 0) pe += (size_t)((naux + ctx->kc_expand - 1) / ctx->kc_expand) * ns * K.nb;
            ex.push_back(g);
            g = GemmDesc{};
            g.A = f32 ? (const void*)K.at32 : (const void*)K.at;
            g.B = K.C;
            g.C = K.Q;
            g.M = at.ma;
            g.K = K.ng;
            g.lda = K.ng;
            g.ldb = K.nb;
            g.ldc = std::max(at.ma, 1);
            g.part_off = pf;
            pf += (size_t)((K.ng + ctx->kc_fwd - 1) / ctx->kc_fwd) * ns * std::max(at.ma, 1);
            fw.push_back(g);
            g = GemmDesc{};
            g.A = f32 ? (const void*)K.caux32 : (const void*)K.caux;
            g.B = K.Y + (size_t)ns * K.nb;
            g.C = K.theta_t;
            g.M = naux;
            g.K = K.nb;
            g.lda = K.nb;
            g.ldb = K.nb;
            g.ldc = naux;
            g.part_off = pp;
            pp += (size_t)((K.nb + ctx->kc_proj - 1) / ctx->kc_proj) * ns * naux;
            pj.push_back(g);
            g = GemmDesc{};
            g.A = K.theta;
            g.B = K.theta_t;
            g.C = K.gram;
            g.M = ns;
            g.K = naux;
            g.lda = naux;
            g.ldb = naux;
            g.ldc = ns;
            g1.push_back(g);
            g.A = K.theta_t;
            g.C = K.gram + (size_t)ns * ns;
            g2.push_back(g);
            g = GemmDesc{};
            g.A = K.evec;
            g.B = K.theta;
            g.C = K.wtmp;
            g.M = naux;
            g.K = naux;
            g.lda = naux;
            g.ldb = naux;
            g.ldc = naux;
            eh.push_back(g);
            g.B = K.wtmp;
            g.C = K.theta;
            en.push_back(g);
        }
        ctx->d_part = dalloc<zd>(ctx, std::max(std::max(pf, pp), pe));
        ctx->gd_expand = upload_descs(ctx, ex);
        ctx->gd_fwd = upload_descs(ctx, fw);
        ctx->gd_proj = upload_descs(ctx, pj);
        ctx->gd_g1 = upload_descs(ctx, g1);
        ctx->gd_g2 = upload_descs(ctx, g2);
        ctx->gd_evh = upload_descs(ctx, eh);
        ctx->gd_evn = upload_descs(ctx, en);
        {
            std::vector<zd*> jm(nk), jv(nk);
            std::vector<double*> jw(nk);
            for (int k = 0; k < nk; ++k) {
                jm[k] = ctx->hkd[k].hsub;
                jv[k] = ctx->hkd[k].evec;
                jw[k] = ctx->hkd[k].eval;
            }
            ctx->d_jac_mats = dupload(ctx, jm.data(), nk);
            ctx->d_jac_vecs = dupload(ctx, jv.data(), nk);
            ctx->d_jac_vals = dupload(ctx, jw.data(), nk);
        }
        // ---- muffin-tin products as batched tiled GEMMs (FP32 forms, many states)
        if (o->precision != RTTDDFT_PREC_FP64 && at.n > 0 && ns >= ZT_MIN_N) {
            ctx->d_mtg = dalloc<zf>(ctx, 5 * ctx->nblk);
            ctx->mtw_stride = 5 * ctx->maxm * ns;
            ctx->mtv_stride = ctx->maxm * ns;
            ctx->d_mtw = dalloc<zd>(ctx, (size_t)nk * at.n * ctx->mtw_stride);
            ctx->d_mtv = dalloc<zd>(ctx, (size_t)nk * at.n * ctx->mtv_stride);
            std::vector<GemmDesc> m1;
            for (int k = 0; k < nk; ++k) {
                for (int al = 0; al < at.n; ++al) {
                    const int m = at.m[al];
                    GemmDesc d{};
                    d.A = ctx->d_mtg + 5 * at.boff[al];
                    d.B = ctx->d_mtv + ((size_t)k * at.n + al) * ctx->mtv_stride;
                    d.C = ctx->d_mtw + ((size_t)k * at.n + al) * ctx->mtw_stride;
                    d.M = 5 * m;
                    d.K = m;
                    d.lda = 5 * m;
                    d.ldb = m;
                    d.ldc = 5 * m;
                    m1.push_back(d);
                }
            }
            ctx->gd_mt1 = upload_descs(ctx, m1);
            if (o->precision == RTTDDFT_PREC_BF16X3 && 2 * ns <= 128 && (long long)nk * at.n <= 65535) {
                // split-BF16 form: the same products as one batch on the tensor cores (one
                // grid slice per (k, atom), within the grid's z limit)
                std::string why;
                const int e = tc_mt_create(&ctx->tcmt, nk, at.n, ctx->maxm, ns, ctx->d_flag, ctx->stream, &why);
                if (e) fail(ctx, e, why);
            }
        }
        {
            StepArgs a = make_args(ctx, 0);
            const int e = prepare_back_kernels(a);
            if (e) fail(ctx, RTTDDFT_ERR_UNSUPPORTED, "table window needs more shared memory than a block has");
            CK(cudaStreamSynchronize(ctx->stream));
            ctx->coop_grid = prepare_cheb_coop(a, ctx->stream, &ctx->cheb_tile);
        }
        // ---- theta(0)
        if (s->c0) {
            size_t c0off = 0;
            for (int k = 0; k < nk; ++k) {
                CK(cudaMemcpy(ctx->hkd[k].C, (const zd*)s->c0 + c0off, (size_t)ctx->nb[k] * ns * sizeof(zd),
                              cudaMemcpyHostToDevice));
                c0off += (size_t)ctx->nb[k] * ns;
            }
            CK(cudaMemset(ctx->d_st, 0, sizeof(DevState)));
            StepArgs a = make_args(ctx, 0);
            StepPlan p = make_plan(ctx);
            launch_operator_pass(a, p, ctx->stream);
            launch_gemm_cn(p.gd_proj, nk, naux, ctx->maxnb, ns, ctx->kc_proj, ctx->d_part, 0, f32, nullptr,
                           ctx->stream);
            launch_split_reduce(p.gd_proj, nk, naux, ns, ctx->kc_proj, ctx->d_part, 0, ctx->stream);
            KCHECK();
            for (int k = 0; k < nk; ++k)
                CK(cudaMemcpyAsync(ctx->hkd[k].theta, ctx->hkd[k].theta_t, (size_t)naux * ns * sizeof(zd),
                                   cudaMemcpyDeviceToDevice, ctx->stream));
        } else {
            std::vector<zd> th((size_t)naux * ns, zmk(0.0, 0.0));
            for (int j = 0; j < ns; ++j) th[j + (size_t)j * naux] = zmk(1.0, 0.0);
            for (int k = 0; k < nk; ++k)
                CK(cudaMemcpy(ctx->hkd[k].theta, th.data(), th.size() * sizeof(zd), cudaMemcpyHostToDevice));
        }
        // ---- ground-state current J(t0) with A = 0
        CK(cudaMemset(ctx->d_st, 0, sizeof(DevState)));
        {
            StepArgs a = make_args(ctx, 0);
            launch_subspace_current(a, 1, ctx->stream);
            KCHECK();
        }
        // ---- Hartree feedback: the potential change is the Hartree potential of
        // the density's change since the start; its interstitial rebuild needs
        // CC_G convolved over N_aux columns and projected
        if (o->hartree) {
            std::string why;
            int e = fft_hartree_init(ctx->fft, s->recip, ctx->vt_dim, ctx->omega, o->hartree_bound, ns, ctx->stream,
                                     &why);
            if (!e) e = fft_reserve_columns(ctx->fft, naux, ctx->stream, &why);
            if (e) fail(ctx, e, why);
            std::vector<GemmDesc> gi;
            std::vector<ToepDesc> td;
            for (int k = 0; k < nk; ++k) {
                KDev& K = ctx->hkd[k];
                K.dvsub = dalloc<zd>(ctx, (size_t)naux * naux);
                zd* T = dalloc<zd>(ctx, (size_t)K.ng * naux);
                td.push_back(ToepDesc{K.caux, T, K.nb, K.ng});
                GemmDesc d{};
                d.A = K.caux;
                d.B = T;
                d.C = K.dvsub;
                d.M = naux;
                d.K = K.ng;
                d.lda = K.nb;
                d.ldb = K.ng;
                d.ldc = naux;
                gi.push_back(d);
            }
            ctx->gd_dvi = upload_descs(ctx, gi);
            ctx->td_dv = dupload(ctx, td.data(), td.size());
            if (f32) {
                // the density is a small change of a large quantity: it is taken from
                // C = CC theta expanded in FP64 (the FP32 expansion's rounding would
                // swamp n(t) - n(0))
                std::vector<GemmDesc> ge;
                std::vector<ToepDesc> tdd;
                for (int k = 0; k < nk; ++k) {
                    KDev& K = ctx->hkd[k];
                    zd* cd = dalloc<zd>(ctx, (size_t)K.nb * ns);
                    GemmDesc g{};
                    g.A = K.caux;
                    g.B = K.theta;
                    g.C = cd;
                    g.M = K.nb;
                    g.K = naux;
                    g.lda = K.nb;
                    g.ldb = naux;
                    g.ldc = K.nb;
                    ge.push_back(g);
                    tdd.push_back(ToepDesc{cd, nullptr, K.nb, K.ng});
                }
                ctx->gd_exp64 = upload_descs(ctx, ge);
                ctx->td_dens = dupload(ctx, tdd.data(), tdd.size());
                // the projection CC_G^H T from the FP32 copy of CC, K slices of 256
                ctx->kc_dvi = 256;
                size_t off = 0;
                std::vector<GemmDesc> g32 = gi;
                for (int k = 0; k < nk; ++k) {
                    g32[k].A = ctx->hkd[k].caux32;
                    g32[k].part_off = off;
                    off += (size_t)((ctx->hkd[k].ng + 255) / 256) * naux * naux;
                }
                ctx->gd_dvi32 = upload_descs(ctx, g32);
                ctx->d_part_dv = dalloc<zd>(ctx, off);
            }
            if (o->hartree_mt_u != 0.0 && at.n > 0) {
                // the muffin-tin part: dh = U (n - n0) per atom, rebuilt into dVV by the
                // four-block form like a prescribed change (s = 1)
                ctx->d_dh = dalloc<zd>(ctx, ctx->nblk);
                CK(cudaMemset(ctx->d_dh, 0, ctx->nblk * sizeof(zd)));
                ctx->d_mtn0 = dalloc<zd>(ctx, ctx->nblk);
                ctx->d_mty = dalloc<zd>(ctx, (size_t)nk * at.lrows * ns);
                ctx->d_mt_lnorm = dalloc<double>(ctx, at.n);
                ctx->d_mt_fn2 = dalloc<double>(ctx, at.n);
                CK(cudaMemset(ctx->d_mt_lnorm, 0, at.n * sizeof(double)));
                CK(cudaMemset(ctx->d_mt_fn2, 0, at.n * sizeof(double)));
                build_mt_rebuild(ctx);
                if (ctx->d_dh32) CK(cudaMemset(ctx->d_dh32, 0, ctx->nblk * sizeof(zf)));
                std::vector<GemmDesc> gy;
                for (int k = 0; k < nk; ++k) {
                    GemmDesc d{};
                    d.A = ctx->hkd[k].lloc;
                    d.B = ctx->hkd[k].theta;
                    d.C = ctx->d_mty + (size_t)k * at.lrows * ns;
                    d.M = at.lrows;
                    d.K = naux;
                    d.lda = at.lrows;
                    d.ldb = naux;
                    d.ldc = at.lrows;
                    gy.push_back(d);
                }
                ctx->gd_mty = upload_descs(ctx, gy);
            }
            CK(cudaMemcpy(ctx->d_kd, ctx->hkd.data(), nk * sizeof(KDev), cudaMemcpyHostToDevice));
            for (int k = 0; k < nk; ++k) ctx->dvnorm[k] = o->hartree_bound;
            ctx->dv_set = true;
            ctx->a_max_cur = -1.0;
            // C(0) = CC theta(0) and the density it carries: the reference of the change
            StepArgs a = make_args(ctx, 0);
            StepPlan p = make_plan(ctx);
            if (p.gd_exp64) {
                launch_gemm_nn(p.gd_exp64, nk, p.maxnb, naux, ns, 0, nullptr, 0, false, nullptr, ctx->stream);
            } else {
                launch_gemm_nn(p.gd_expand, nk, p.maxnb, naux, ns, p.kc_expand, p.kc_expand > 0 ? p.part : nullptr, 0,
                               f32, nullptr, ctx->stream);
                if (p.kc_expand > 0)
                    launch_split_reduce(p.gd_expand, nk, p.maxnb, ns, p.kc_expand, p.part, 0, ctx->stream);
            }
            launch_fft_density(ctx->fft, p.td_dens, nk, ns, a.occ, a.wk, 1, ctx->stream);
            if (ctx->d_mtn0) {
                // the reference muffin-tin densities of theta(0) and the bound's factors
                launch_mt_feedback(a, p, 1, nullptr, ctx->stream);
                launch_mt_lnorm(a, ctx->stream);
            }
            KCHECK();
        }
        CK(cudaStreamSynchronize(ctx->stream));
        *out = ctx;
        return RTTDDFT_OK;
    } catch (Fail& f) {
        if (ctx) {
            g_last_error = ctx->err;
            rttddft_destroy(ctx);
        }
        return f.code;
    }
}

// Chebyshev scaling [lam_c - lam_h, lam_c + lam_h] containing the spectrum of
// HH(t) = diag(eps) + (A/c).PP + |A|^2/(2c^2) + s dVV_1 for every |A| <= a_max
// and |s| <= s_max: ||sum_l (A_l/c) PP_l||_2 <= |A| sum_l ||PP_l||_F / c.
// The coefficients are rebuilt on the device only when the bounds grow.
static void ensure_interval(rttddft_ctx* ctx, double a_need, double s_need) {
    if (ctx->a_max_cur >= 0.0 && a_need <= ctx->a_max_cur && s_need <= ctx->s_max_cur) return;
    const double amax = std::max(a_need, std::max(ctx->a_max_cur, 0.0));
    const double smax = std::max(s_need, std::max(ctx->s_max_cur, 0.0));
    const int nk = ctx->nk;
    const double c = ctx->c, dt = ctx->opt.dt;
    std::vector<double> lam(LAM_N * nk, 0.0);
    double zmax = 0.0;
    for (int k = 0; k < nk; ++k) {
        const double bl = amax * (ctx->pnorm[3 * k] + ctx->pnorm[3 * k + 1] + ctx->pnorm[3 * k + 2]) / c;
        const double a2 = amax * amax / (2 * c * c);
        const double sd = smax * ctx->dvnorm[k];
        double lo = ctx->eps_min[k] - bl - sd;
        double hi = ctx->eps_max[k] + bl + a2 + sd;
        const double pad = 1e-10 * std::max(1.0, std::max(fabs(lo), fabs(hi)));
        lo -= pad;
        hi += pad;
        lam[LAM_N * k] = 0.5 * (hi + lo);
        lam[LAM_N * k + 1] = std::max(0.5 * (hi - lo), 1e-12);
        lam[LAM_N * k + 2] = 1.0 / lam[LAM_N * k + 1];
        lam[LAM_N * k + 3] = cos(-dt * lam[LAM_N * k]);
        lam[LAM_N * k + 4] = sin(-dt * lam[LAM_N * k]);
        zmax = std::max(zmax, dt * lam[LAM_N * k + 1]);
    }
    const double tol = ctx->opt.cheb_tol > 0 ? ctx->opt.cheb_tol : 1e-16;
    int nt;
    if (ctx->opt.propagator == RTTDDFT_PROP_CN) {
        // Cayley map: pole of 1/(1 + i dt/2 lam) at lam = 2i/dt; coefficients
        // decay like rho^-n with rho the Bernstein ellipse through the pole
        double nmax = 3;
        for (int k = 0; k < nk; ++k) {
            const cplx xp = (cplx(0.0, 2.0 / dt) - lam[LAM_N * k]) / lam[LAM_N * k + 1];
            cplx r = xp + std::sqrt(xp * xp - 1.0);
            if (std::abs(r) < 1.0) r = xp - std::sqrt(xp * xp - 1.0);
            nmax = std::max(nmax, log(1e-2 * tol) / -log(std::abs(r)) + 4);
        }
        nt = (int)ceil(nmax);
        if (nt > 120) fail(ctx, RTTDDFT_ERR_UNSUPPORTED, "Crank-Nicolson series too long for this dt and spectrum");
    } else {
        // |J_n(z)| <= (z/2)^n / n!: stop once 2 (z/2)^n / n! < tol/100 with n > z
        double term = 1.0;
        int n = 1;
        for (; n < RTD_MAX_TERMS - 3; ++n) {
            term *= (0.5 * zmax) / n;
            if (n > zmax && 2.0 * term < 1e-2 * tol) break;
        }
        nt = n + 2;
    }
    ctx->nterms = std::max(3, std::min(nt, RTD_MAX_TERMS));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(ctx->d_lam, lam.data(), lam.size() * sizeof(double), cudaMemcpyHostToDevice));
    StepArgs a = make_args(ctx, 0);
    launch_prep_coef(a, ctx->stream);
    KCHECK();
    ctx->a_max_cur = amax;
    ctx->s_max_cur = smax;
}

static void ensure_call_cap(rttddft_ctx* ctx, int nsteps) {
    if (nsteps <= ctx->call_cap) return;
    CK(cudaStreamSynchronize(ctx->stream));
    dfree(ctx, ctx->d_a);
    dfree(ctx, ctx->d_dvs);
    ctx->call_cap = nsteps;
    ctx->d_a = dalloc<double>(ctx, 3 * (size_t)nsteps);
    ctx->d_dvs = dalloc<double>(ctx, (size_t)nsteps);
    if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
        ctx->g_key_nterms = -1;
    }
}

static void run_steps(rttddft_ctx* ctx, int nsteps, int dv_on) {
    StepArgs a = make_args(ctx, dv_on);
    StepPlan p = make_plan(ctx);
    CK(cudaMemsetAsync(&ctx->d_st->cstep, 0, sizeof(int), ctx->stream));
    const int G = ctx->opt.graph_steps;
    int done = 0;
    if (G > 0 && nsteps >= G) {
        if (!ctx->gexec || ctx->g_key_nterms != ctx->nterms || ctx->g_key_dv != dv_on || ctx->g_key_steps != G) {
            if (ctx->gexec) {
                CK(cudaStreamSynchronize(ctx->stream));
                cudaGraphExecDestroy(ctx->gexec);
                ctx->gexec = nullptr;
            }
            cudaGraph_t graph;
            CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
            for (int i = 0; i < G; ++i) launch_step(a, p, ctx->stream, &ctx->launches_per_step);
            cudaError_t e1 = cudaGetLastError();
            cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &graph);
            if (e1 != cudaSuccess || e2 != cudaSuccess) {
                set_err(ctx, std::string("graph capture failed: ") + cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
                throw Fail{RTTDDFT_ERR_CUDA};
            }
            CK(cudaGraphInstantiate(&ctx->gexec, graph, 0));
            cudaGraphDestroy(graph);
            ctx->g_key_nterms = ctx->nterms;
            ctx->g_key_dv = dv_on;
            ctx->g_key_steps = G;
        }
        while (nsteps - done >= G) {
            CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
            done += G;
        }
    }
    for (; done < nsteps; ++done) launch_step(a, p, ctx->stream, &ctx->launches_per_step);
    KCHECK();
}

// Wait for the device and turn a raised device flag into an error code.
static void sync_and_check(rttddft_ctx* ctx) {
    CK(cudaStreamSynchronize(ctx->stream));
    int flag = 0;
    CK(cudaMemcpy(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        CK(cudaMemset(ctx->d_flag, 0, sizeof(int)));
        if (flag & 1) fail(ctx, RTTDDFT_ERR_TIMEOUT, "Jacobi eigensolver reached its sweep limit");
        if (flag & 4) fail(ctx, RTTDDFT_ERR_TIMEOUT, "the grid barrier of the Chebyshev series timed out");
        if (flag & 8) fail(ctx, RTTDDFT_ERR_TIMEOUT, "a tensor-core pipeline wait timed out");
        if (flag & 32)
            fail(ctx, RTTDDFT_ERR_NONFINITE, "a scaled operand of the split-FP16 form left the fp16 range");
        if (flag & 64)
            fail(ctx, RTTDDFT_ERR_ARG, "the Hartree potential change exceeded hartree_bound (the spectral interval)");
        fail(ctx, RTTDDFT_ERR_ARG, "a pulse sample or dv scale exceeded a_max / s_max");
    }
}

static void stage_host(rttddft_ctx* ctx, const double* src, size_t n, double* dst_dev) {
    if (ctx->stage_ev) CK(cudaEventSynchronize(ctx->stage_ev));
    if ((int)n > ctx->stage_cap) {
        if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
        ctx->h_stage = nullptr;
        CK(cudaMallocHost(&ctx->h_stage, n * sizeof(double)));
        ctx->stage_cap = (int)n;
    }
    if (!ctx->stage_ev) CK(cudaEventCreateWithFlags(&ctx->stage_ev, cudaEventDisableTiming));
    memcpy(ctx->h_stage, src, n * sizeof(double));
    CK(cudaMemcpyAsync(dst_dev, ctx->h_stage, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaEventRecord(ctx->stage_ev, ctx->stream));
}

int rttddft_step(rttddft_ctx* ctx, int nsteps, const double* a_samples, const double* dv_scale) {
    if (!ctx) return RTTDDFT_ERR_ARG;
    try {
        if (nsteps < 1 || !a_samples) fail(ctx, RTTDDFT_ERR_ARG, "nsteps < 1 or a_samples NULL");
        if (ctx->rec_count + nsteps > ctx->opt.max_record)
            fail(ctx, RTTDDFT_ERR_ARG, "record capacity exceeded: call rttddft_observables with clear");
        if (dv_scale && !ctx->dv_set) fail(ctx, RTTDDFT_ERR_ARG, "dv_scale given before rttddft_set_dv");
        if (dv_scale && ctx->opt.hartree)
            fail(ctx, RTTDDFT_ERR_ARG, "dv_scale is not taken with the Hartree feedback (the density sets the change)");
        {
            int flag = 0;  // errors raised by earlier, finished work
            if (cudaStreamQuery(ctx->stream) == cudaSuccess) {
                CK(cudaMemcpy(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost));
                if (flag) sync_and_check(ctx);
            } else {
                cudaGetLastError();
            }
        }
        ensure_call_cap(ctx, nsteps);
        const size_t na = 3 * (size_t)nsteps;
        double a_need = 0.0, s_need = 0.0;
        const bool a_dev = is_device_ptr(a_samples);
        const bool s_dev = dv_scale && is_device_ptr(dv_scale);
        std::vector<double> tmp;
        if (a_dev) {
            CK(cudaMemcpyAsync(ctx->d_a, a_samples, na * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
            if (ctx->opt.a_max > 0) {
                a_need = ctx->opt.a_max;
            } else {
                tmp.resize(na);
                CK(cudaMemcpyAsync(tmp.data(), a_samples, na * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
                CK(cudaStreamSynchronize(ctx->stream));
            }
        } else {
            if (!finite_all(a_samples, na)) fail(ctx, RTTDDFT_ERR_NONFINITE, "a_samples not finite");
            tmp.assign(a_samples, a_samples + na);
        }
        for (size_t i = 0; i + 2 < tmp.size(); i += 3)
            a_need = std::max(a_need, sqrt(tmp[i] * tmp[i] + tmp[i + 1] * tmp[i + 1] + tmp[i + 2] * tmp[i + 2]));
        if (!a_dev && ctx->opt.a_max > 0) {
            if (a_need > ctx->opt.a_max) fail(ctx, RTTDDFT_ERR_ARG, "|A_k| exceeds a_max");
            a_need = ctx->opt.a_max;
        }
        std::vector<double> stmp;
        if (dv_scale) {
            if (s_dev) {
                CK(cudaMemcpyAsync(ctx->d_dvs, dv_scale, nsteps * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
                if (ctx->opt.s_max > 0) {
                    s_need = ctx->opt.s_max;
                } else {
                    stmp.resize(nsteps);
                    CK(cudaMemcpyAsync(stmp.data(), dv_scale, nsteps * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
                    CK(cudaStreamSynchronize(ctx->stream));
                }
            } else {
                if (!finite_all(dv_scale, nsteps)) fail(ctx, RTTDDFT_ERR_NONFINITE, "dv_scale not finite");
                stmp.assign(dv_scale, dv_scale + nsteps);
            }
            for (double x : stmp) s_need = std::max(s_need, fabs(x));
            if (!s_dev && ctx->opt.s_max > 0) {
                if (s_need > ctx->opt.s_max) fail(ctx, RTTDDFT_ERR_ARG, "|s_k| exceeds s_max");
                s_need = ctx->opt.s_max;
            }
        }
        if (ctx->opt.hartree) s_need = 1.0;  // dVV = 1 x the Hartree change, bounded by hartree_bound
        ensure_interval(ctx, a_need, s_need);
        if (!a_dev) stage_host(ctx, a_samples, na, ctx->d_a);
        if (dv_scale && !s_dev) {
            // second staging: wait for the first copy before reusing the buffer
            stage_host(ctx, dv_scale, nsteps, ctx->d_dvs);
        }
        if ((a_dev && ctx->opt.a_max > 0) || (s_dev && ctx->opt.s_max > 0))
            launch_check_samples(ctx->d_a, a_dev ? nsteps : 0, ctx->a_max_cur, ctx->d_dvs,
                                 s_dev ? nsteps : 0, ctx->s_max_cur, ctx->d_flag, ctx->stream);
        run_steps(ctx, nsteps, (dv_scale || ctx->opt.hartree) ? 1 : 0);
        ctx->rec_count += nsteps;
        ctx->steps_done += nsteps;
        ctx->time += nsteps * ctx->opt.dt;
        return RTTDDFT_OK;
    } catch (Fail& f) {
        return f.code;
    }
}

int rttddft_observables(rttddft_ctx* ctx, rttddft_obs* out, int clear) {
    if (!ctx || !out) return RTTDDFT_ERR_ARG;
    try {
        sync_and_check(ctx);
        const int n = ctx->rec_count;
        if (out->capacity < n) fail(ctx, RTTDDFT_ERR_ARG, "observable capacity smaller than the records held");
        std::vector<double> r((size_t)n * RTD_REC_STRIDE);
        if (n) CK(cudaMemcpy(r.data(), ctx->d_rec, r.size() * sizeof(double), cudaMemcpyDeviceToHost));
        for (int i = 0; i < n; ++i) {
            const double* q = r.data() + (size_t)i * RTD_REC_STRIDE;
            if (out->t) out->t[i] = q[REC_T];
            for (int l = 0; l < 3; ++l) {
                if (out->j) out->j[3 * i + l] = q[REC_J + l];
                if (out->j_full) out->j_full[3 * i + l] = q[REC_JF + l];
                if (out->dmu) out->dmu[3 * i + l] = q[REC_DMU + l];
            }
            if (out->energy) out->energy[i] = q[REC_E];
            if (out->norm_dev) out->norm_dev[i] = q[REC_NDEV];
            if (out->resid) out->resid[i] = q[REC_RES];
            if (out->dt_cr) out->dt_cr[i] = q[REC_DTCR];
            if (out->n_exc) out->n_exc[i] = q[REC_NEXC];
        }
        out->count = n;
        if (clear) {
            CK(cudaMemsetAsync(&ctx->d_st->rec_count, 0, sizeof(int), ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            ctx->rec_count = 0;
        }
        return RTTDDFT_OK;
    } catch (Fail& f) {
        return f.code;
    }
}

int rttddft_get_state(rttddft_ctx* ctx, int k, double* theta, double* c) {
    if (!ctx) return RTTDDFT_ERR_ARG;
    try {
        if (k < 0 || k >= ctx->nk) fail(ctx, RTTDDFT_ERR_ARG, "k out of range");
        sync_and_check(ctx);
        const KDev& K = ctx->hkd[k];
        if (theta)
            CK(cudaMemcpy(theta, K.theta, (size_t)ctx->naux * ctx->ns * sizeof(zd), cudaMemcpyDeviceToHost));
        if (c) {
            launch_gemm_nn(ctx->gd_expand, ctx->nk, ctx->maxnb, ctx->naux, ctx->ns, 0, nullptr, 0,
                           ctx->opt.precision != RTTDDFT_PREC_FP64, nullptr, ctx->stream);
            KCHECK();
            CK(cudaStreamSynchronize(ctx->stream));
            CK(cudaMemcpy(c, K.C, (size_t)K.nb * ctx->ns * sizeof(zd), cudaMemcpyDeviceToHost));
        }
        return RTTDDFT_OK;
    } catch (Fail& f) {
        return f.code;
    }
}

int rttddft_set_state(rttddft_ctx* ctx, int k, const double* theta) {
    if (!ctx) return RTTDDFT_ERR_ARG;
    try {
        if (k < 0 || k >= ctx->nk || !theta) fail(ctx, RTTDDFT_ERR_ARG, "k out of range or theta NULL");
        if (!finite_all(theta, 2 * (size_t)ctx->naux * ctx->ns)) fail(ctx, RTTDDFT_ERR_NONFINITE, "theta not finite");
        CK(cudaStreamSynchronize(ctx->stream));
        CK(cudaMemcpy(ctx->hkd[k].theta, theta, (size_t)ctx->naux * ctx->ns * sizeof(zd), cudaMemcpyHostToDevice));
        return RTTDDFT_OK;
    } catch (Fail& f) {
        return f.code;
    }
}

int rttddft_get_aux(rttddft_ctx* ctx, int k, double* caux, double* eps, double* pp) {
    if (!ctx) return RTTDDFT_ERR_ARG;
    try {
        if (k < 0 || k >= ctx->nk) fail(ctx, RTTDDFT_ERR_ARG, "k out of range");
        CK(cudaStreamSynchronize(ctx->stream));
        const KDev& K = ctx->hkd[k];
        const size_t nn = (size_t)ctx->naux * ctx->naux;
        if (caux) CK(cudaMemcpy(caux, K.caux, (size_t)K.nb * ctx->naux * sizeof(zd), cudaMemcpyDeviceToHost));
        if (eps) CK(cudaMemcpy(eps, K.eps, ctx->naux * sizeof(double), cudaMemcpyDeviceToHost));
        if (pp) CK(cudaMemcpy(pp, K.psub, 3 * nn * sizeof(zd), cudaMemcpyDeviceToHost));
        return RTTDDFT_OK;
    } catch (Fail& f) {
        return f.code;
    }
}

int rttddft_get_info(rttddft_ctx* ctx, rttddft_info* info) {
    if (!ctx || !info) return RTTDDFT_ERR_ARG;
    info->steps_done = ctx->steps_done;
    info->time = ctx->time;
    info->n_basis_max = ctx->maxnb;
    info->cheb_terms = ctx->nterms;
    info->dt_cr0 = ctx->dtcr0;
    info->kernel_launches_per_step = ctx->launches_per_step;
    info->precision = ctx->opt.precision;
    int v[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (ctx->tc) tc_plan_info(ctx->tc, v);
    info->tc_candidates = v[6];
    info->tc_interstitial_ns = v[7];
    info->tc_matching_ns = v[8];
    info->tc_tile_n = v[0];
    info->tc_stages = v[1];
    info->tc_kblocks = v[2];
    info->tc_slices = v[3];
    info->tc_window = v[4];
    info->tc_smem = v[5];
    info->tc_gen_threads = v[9];
    info->tc_a_tmem = v[10];
    info->tc_back_parts = v[11];
    info->interstitial = ctx->opt.interstitial;
    fft_plan_info(ctx->fft, info->fft_grid, &info->fft_fused);
    return RTTDDFT_OK;
}

}  // extern "C"

// The muffin-tin four blocks of the potential-change rebuild (Eq. v_MT):
// W = dh L per atom and dVV = L^H W per k-point, with L the atoms' rows of the
// local coordinates of CC; FP32 copies of dh and L for the reduced-precision
// forms.  Allocates the per-k W buffers; d_dh and the K.dvsub must exist.
static void build_mt_rebuild(rttddft_ctx* ctx) {
    const AtomTab& at = ctx->at;
    const int nk = ctx->nk, naux = ctx->naux;
    size_t nblk = 0;
    for (int a = 0; a < at.n; ++a) nblk += (size_t)at.m[a] * at.m[a];
    std::vector<GemmDesc> w, g;
    for (int k = 0; k < nk; ++k) {
        KDev& K = ctx->hkd[k];
        zd* W = dalloc<zd>(ctx, (size_t)std::max(at.lrows, 1) * naux);
        for (int a = 0; a < at.n; ++a) {
            GemmDesc d{};
            d.A = ctx->d_dh + at.boff[a];
            d.B = K.lloc + at.loff[a];
            d.C = W + at.loff[a];
            d.M = at.m[a];
            d.K = at.m[a];
            d.lda = at.m[a];
            d.ldb = at.lrows;
            d.ldc = at.lrows;
            w.push_back(d);
        }
        GemmDesc d{};
        d.A = K.lloc;
        d.B = W;
        d.C = K.dvsub;
        d.M = naux;
        d.K = at.lrows;
        d.lda = std::max(at.lrows, 1);
        d.ldb = std::max(at.lrows, 1);
        d.ldc = naux;
        g.push_back(d);
    }
    ctx->gd_dvw = upload_descs(ctx, w);
    ctx->gd_dvg = upload_descs(ctx, g);
    if (ctx->opt.precision != RTTDDFT_PREC_FP64 && at.n > 0) {
        // reduced-precision forms: W = (s dh) L and L^H W on the FP32 tiled
        // kernels, from FP32 copies of dh and of the local coordinates L
        ctx->d_dh32 = dalloc<zf>(ctx, nblk);
        std::vector<GemmDesc> w32 = w, g32 = g;
        for (auto& d : w32) d.A = ctx->d_dh32 + ((const zd*)d.A - ctx->d_dh);
        for (int k = 0; k < nk; ++k) {
            zf* l32 = dalloc<zf>(ctx, (size_t)at.lrows * naux);
            launch_convert_f32(ctx->hkd[k].lloc, l32, (size_t)at.lrows * naux, ctx->stream);
            g32[k].A = l32;
        }
        ctx->gd_dvw32 = upload_descs(ctx, w32);
        ctx->gd_dvg32 = upload_descs(ctx, g32);
    }
}

extern "C" {

int rttddft_set_dv(rttddft_ctx* ctx, const double* dh, const double* dvtab) {
    if (!ctx) return RTTDDFT_ERR_ARG;
    try {
        if (ctx->opt.hartree) fail(ctx, RTTDDFT_ERR_ARG, "with the Hartree feedback the potential change comes from the density");
        const AtomTab& at = ctx->at;
        size_t nblk = 0;
        for (int a = 0; a < at.n; ++a) nblk += (size_t)at.m[a] * at.m[a];
        if ((at.n > 0 && !dh) || !dvtab) fail(ctx, RTTDDFT_ERR_ARG, "dh or dvtab NULL");
        if ((at.n > 0 && !finite_all(dh, 2 * nblk)) || !finite_all(dvtab, 2 * (size_t)ctx->nvt))
            fail(ctx, RTTDDFT_ERR_NONFINITE, "dh or dvtab not finite");
        for (int a = 0; a < at.n; ++a)
            if (herm_dev(dh + 2 * at.boff[a], at.m[a]) > 1e-12)
                fail(ctx, RTTDDFT_ERR_NOT_HERMITIAN, "dh block not Hermitian");
        {
            const cplx* V = (const cplx*)dvtab;
            double dev = 0.0, mx = 1e-300;
            for (int i = 0; i < ctx->nvt; ++i) mx = std::max(mx, std::abs(V[i]));
            for (int i = 0; i < ctx->nvt; ++i) dev = std::max(dev, std::abs(V[i] - std::conj(V[ctx->nvt - 1 - i])));
            if (dev > 1e-12 * mx) fail(ctx, RTTDDFT_ERR_NOT_HERMITIAN, "dvtab not Hermitian in g");
        }
        const int nk = ctx->nk, naux = ctx->naux;
        CK(cudaStreamSynchronize(ctx->stream));
        if (!ctx->dv_set) {
            if (at.n > 0) ctx->d_dh = dalloc<zd>(ctx, nblk);
            ctx->d_dvtab = dalloc<zd>(ctx, ctx->nvt);
            ctx->d_vstep = dalloc<zd>(ctx, ctx->nvt);
            if (ctx->opt.precision != RTTDDFT_PREC_FP64) ctx->d_vstep32 = dalloc<zf>(ctx, ctx->nvt);
            if (ctx->opt.precision >= RTTDDFT_PREC_BF16X3) ctx->d_vsteps = dalloc<uint2>(ctx, ctx->nvt);
            std::vector<GemmDesc> gi;
            std::vector<ToepDesc> td;
            for (int k = 0; k < nk; ++k) {
                KDev& K = ctx->hkd[k];
                K.dvsub = dalloc<zd>(ctx, (size_t)naux * naux);
                zd* T = dalloc<zd>(ctx, (size_t)K.ng * naux);
                td.push_back(ToepDesc{K.caux, T, K.nb, K.ng});
                GemmDesc d{};
                d.A = K.caux;
                d.B = T;
                d.C = K.dvsub;
                d.M = naux;
                d.K = K.ng;
                d.lda = K.nb;
                d.ldb = K.ng;
                d.ldc = naux;
                gi.push_back(d);
            }
            build_mt_rebuild(ctx);
            ctx->gd_dvi = upload_descs(ctx, gi);
            ctx->td_dv = dupload(ctx, td.data(), td.size());
            if (ctx->tc && !ctx->fft) {
                // tensor-core forms: the interstitial convolution on tcgen05
                std::vector<const zd*> cp(nk);
                std::vector<int> nbv(nk), ngv(nk);
                for (int k = 0; k < nk; ++k) {
                    cp[k] = ctx->hkd[k].caux;
                    nbv[k] = ctx->hkd[k].nb;
                    ngv[k] = ctx->hkd[k].ng;
                }
                std::string why;
                const int e = tc_dv_prepare(ctx->tc, cp.data(), nbv.data(), ngv.data(), naux, ctx->nvt,
                                            ctx->stream, &why);
                if (e) fail(ctx, e, why);
            }
            if (ctx->opt.precision != RTTDDFT_PREC_FP64) {
                // reduced-precision forms: the projection CC_G^H T from the FP32 copy of CC
                // in K slices of 256, FP64 sums of the slices
                ctx->kc_dvi = 256;
                size_t off = 0;
                std::vector<GemmDesc> g32 = gi;
                for (int k = 0; k < nk; ++k) {
                    g32[k].A = ctx->hkd[k].caux32;
                    g32[k].part_off = off;
                    off += (size_t)((ctx->hkd[k].ng + 255) / 256) * naux * naux;
                }
                ctx->gd_dvi32 = upload_descs(ctx, g32);
                ctx->d_part_dv = dalloc<zd>(ctx, off);
            }
            CK(cudaMemcpy(ctx->d_kd, ctx->hkd.data(), nk * sizeof(KDev), cudaMemcpyHostToDevice));
        }
        if (at.n > 0) CK(cudaMemcpy(ctx->d_dh, dh, nblk * sizeof(zd), cudaMemcpyHostToDevice));
        if (ctx->d_dh32) launch_convert_f32(ctx->d_dh, ctx->d_dh32, nblk, ctx->stream);
        CK(cudaMemcpy(ctx->d_dvtab, dvtab, ctx->nvt * sizeof(zd), cudaMemcpyHostToDevice));
        if (ctx->tc && !ctx->fft) {
            double vmax = 0.0;
            for (int i = 0; i < 2 * ctx->nvt; ++i) vmax = std::max(vmax, std::fabs(dvtab[i]));
            tc_dv_set_table(ctx->tc, ctx->d_dvtab, ctx->nvt, vmax, ctx->stream);
        }
        if (ctx->fft) {
            std::string why;
            const int e = fft_set_dv(ctx->fft, ctx->d_dvtab, ctx->vt_dim, naux, ctx->stream, &why);
            if (e) fail(ctx, e, why);
            KCHECK();
        }
        ctx->dv_set = true;
        // bound || CC^H dV_1 CC ||_F for the Chebyshev scaling (one evaluation with s = 1)
        {
            const double one = 1.0;
            CK(cudaMemcpy(&ctx->d_st->cur_s, &one, sizeof(double), cudaMemcpyHostToDevice));
            StepArgs a = make_args(ctx, 1);
            StepPlan p = make_plan(ctx);
            if (at.n > 0) {
                launch_gemm_nn(p.gd_dvw, p.n_dvw, p.maxm, p.maxm, naux, 0, nullptr, 0, false, &a.st->cur_s, ctx->stream);
                launch_gemm_cn(p.gd_dvg, nk, naux, at.lrows, naux, 0, nullptr, 0, false, nullptr, ctx->stream);
            } else {
                for (int k = 0; k < nk; ++k) launch_zero(ctx->hkd[k].dvsub, (size_t)naux * naux, ctx->stream);
            }
            launch_toeplitz(ctx->d_kd, p.td_dv, nk, ctx->maxng, naux, ctx->d_dvtab, ctx->vt_center, 0, 0,
                            &a.st->cur_s, ctx->stream);
            launch_gemm_cn(p.gd_dvi, nk, naux, ctx->maxng, naux, 0, nullptr, 1, false, nullptr, ctx->stream);
            KCHECK();
            CK(cudaStreamSynchronize(ctx->stream));
            for (int k = 0; k < nk; ++k) {
                std::vector<double> v(2 * (size_t)naux * naux);
                CK(cudaMemcpy(v.data(), ctx->hkd[k].dvsub, v.size() * sizeof(double), cudaMemcpyDeviceToHost));
                double f = 0.0;
                for (double x : v) f += x * x;
                ctx->dvnorm[k] = sqrt(f);
            }
            ctx->a_max_cur = -1.0;  // the spectral interval depends on ||dVV_1||
        }
        return RTTDDFT_OK;
    } catch (Fail& f) {
        return f.code;
    }
}

int rttddft_apply(rttddft_ctx* ctx, int k, int ncols, const double* x, const double* a_vec,
                  double dv_scale, double* hx, double* sx) {
    if (!ctx) return RTTDDFT_ERR_ARG;
    try {
        if (k < 0 || k >= ctx->nk || ncols < 1 || !x || !a_vec || !hx || !sx)
            fail(ctx, RTTDDFT_ERR_ARG, "bad argument to rttddft_apply");
        if (dv_scale != 0.0 && !ctx->dv_set) fail(ctx, RTTDDFT_ERR_ARG, "dv_scale != 0 before rttddft_set_dv");
        CK(cudaStreamSynchronize(ctx->stream));
        const bool dev = is_device_ptr(x);
        const cudaMemcpyKind kin = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        const cudaMemcpyKind kout = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        const KDev& K = ctx->hkd[k];
        const int ns = ctx->ns, nb = K.nb;
        DevState hst{};
        CK(cudaMemcpy(&hst, ctx->d_st, sizeof(DevState), cudaMemcpyDeviceToHost));
        DevState tmp = hst;
        for (int l = 0; l < 3; ++l) tmp.cur_a[l] = a_vec[l];
        tmp.cur_s = dv_scale;
        tmp.cur_aa = (a_vec[0] * a_vec[0] + a_vec[1] * a_vec[1] + a_vec[2] * a_vec[2]) / (2 * ctx->c * ctx->c);
        CK(cudaMemcpy(ctx->d_st, &tmp, sizeof(DevState), cudaMemcpyHostToDevice));
        const int dv_on = (dv_scale != 0.0) ? 1 : 0;
        StepArgs a = make_args(ctx, dv_on);
        a.kd = ctx->d_kd + k;
        a.nk = 1;
        a.kofs = k;
        StepPlan p = make_plan(ctx);
        p.gd_fwd = ctx->gd_fwd + k;
        if (p.gd_mt1) p.gd_mt1 = ctx->gd_mt1 + (size_t)k * ctx->at.n;
        p.maxng = K.ng;
        if (dv_on && !ctx->opt.hartree) launch_vstep(a, ctx->stream);
        const zd* xz = (const zd*)x;
        zd* hz = (zd*)hx;
        zd* sz = (zd*)sx;
        for (int c0 = 0; c0 < ncols; c0 += ns) {
            const int w = std::min(ns, ncols - c0);
            if (w < ns) launch_zero(K.C, (size_t)nb * ns, ctx->stream);
            CK(cudaMemcpyAsync(K.C, xz + (size_t)c0 * nb, (size_t)w * nb * sizeof(zd), kin, ctx->stream));
            launch_operator_pass(a, p, ctx->stream);
            KCHECK();
            CK(cudaMemcpyAsync(hz + (size_t)c0 * nb, K.Y, (size_t)w * nb * sizeof(zd), kout, ctx->stream));
            CK(cudaMemcpyAsync(sz + (size_t)c0 * nb, K.Y + (size_t)ns * nb, (size_t)w * nb * sizeof(zd), kout,
                               ctx->stream));
            sync_and_check(ctx);
        }
        CK(cudaMemcpy(ctx->d_st, &hst, sizeof(DevState), cudaMemcpyHostToDevice));
        return RTTDDFT_OK;
    } catch (Fail& f) {
        return f.code;
    }
}

int rttddft_trace_steps(rttddft_ctx* ctx, int nsteps, const double* a_samples, const double* dv_scale,
                        rttddft_trace* out) {
    if (!ctx) return RTTDDFT_ERR_ARG;
    std::vector<cudaEvent_t> ev;
    try {
        if (!out || !out->names || !out->ms || out->capacity < 1 || nsteps < 1 || !a_samples)
            fail(ctx, RTTDDFT_ERR_ARG, "bad argument to rttddft_trace_steps");
        if (ctx->rec_count + nsteps > ctx->opt.max_record)
            fail(ctx, RTTDDFT_ERR_ARG, "record capacity exceeded: call rttddft_observables with clear");
        if (dv_scale && !ctx->dv_set) fail(ctx, RTTDDFT_ERR_ARG, "dv_scale given before rttddft_set_dv");
        if (dv_scale && ctx->opt.hartree)
            fail(ctx, RTTDDFT_ERR_ARG, "dv_scale is not taken with the Hartree feedback (the density sets the change)");
        sync_and_check(ctx);
        ensure_call_cap(ctx, nsteps);
        const size_t na = 3 * (size_t)nsteps;
        double a_need = 0.0, s_need = 0.0;
        for (size_t i = 0; i < na; i += 3)
            a_need = std::max(a_need, sqrt(a_samples[i] * a_samples[i] + a_samples[i + 1] * a_samples[i + 1] +
                                           a_samples[i + 2] * a_samples[i + 2]));
        if (ctx->opt.a_max > 0) a_need = std::max(a_need, ctx->opt.a_max);
        if (dv_scale) {
            for (int i = 0; i < nsteps; ++i) s_need = std::max(s_need, fabs(dv_scale[i]));
            if (ctx->opt.s_max > 0) s_need = std::max(s_need, ctx->opt.s_max);
        }
        if (ctx->opt.hartree) s_need = 1.0;
        ensure_interval(ctx, a_need, s_need);
        CK(cudaMemcpy(ctx->d_a, a_samples, na * sizeof(double), cudaMemcpyHostToDevice));
        if (dv_scale) CK(cudaMemcpy(ctx->d_dvs, dv_scale, nsteps * sizeof(double), cudaMemcpyHostToDevice));
        const int dv_on = (dv_scale || ctx->opt.hartree) ? 1 : 0;
        StepArgs a = make_args(ctx, dv_on);
        StepPlan p = make_plan(ctx);
        CK(cudaMemsetAsync(&ctx->d_st->cstep, 0, sizeof(int), ctx->stream));
        const int cap = 256;
        ev.resize(cap + 1);
        for (auto& e : ev) CK(cudaEventCreate(&e));
        std::vector<const char*> names(cap);
        std::vector<double> acc(cap, 0.0);
        int slots = 0;
        // one step with an event after every launch, captured in a graph so that
        // the events measure device time without host launch gaps
        TraceHook tr{ev.data() + 1, names.data(), 0, cap};
        cudaGraph_t graph;
        cudaGraphExec_t gx = nullptr;
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        CK(cudaEventRecordWithFlags(ev[0], ctx->stream, cudaEventRecordExternal));
        launch_step(a, p, ctx->stream, &ctx->launches_per_step, &tr);
        {
            cudaError_t e1 = cudaGetLastError();
            cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &graph);
            if (e1 != cudaSuccess || e2 != cudaSuccess) fail(ctx, RTTDDFT_ERR_CUDA, "trace graph capture failed");
        }
        CK(cudaGraphInstantiate(&gx, graph, 0));
        cudaGraphDestroy(graph);
        for (int i = 0; i < nsteps; ++i) {
            CK(cudaGraphLaunch(gx, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            for (int j = 0; j < tr.n; ++j) {
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, ev[j], ev[j + 1]));
                acc[j] += ms;
            }
            slots = tr.n;
        }
        cudaGraphExecDestroy(gx);
        const int n = std::min(slots, out->capacity);
        for (int j = 0; j < n; ++j) {
            out->names[j] = names[j];
            out->ms[j] = acc[j];
        }
        out->count = n;
        for (auto& e : ev) cudaEventDestroy(e);
        ctx->rec_count += nsteps;
        ctx->steps_done += nsteps;
        ctx->time += nsteps * ctx->opt.dt;
        return RTTDDFT_OK;
    } catch (Fail& f) {
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        return f.code;
    }
}

int rttddft_adjoint(rttddft_ctx* ctx, int nsteps, const double* a_samples, const double* dv_scale,
                    const double* gdir, int ckpt_every, double* grad, double* dmu_out) {
    if (!ctx) return RTTDDFT_ERR_ARG;
    std::vector<void*> tmp;
    DevState saved{};
    std::vector<zd*> theta_saved;
    bool restore = false;
    try {
        if (ctx->opt.hartree)
            fail(ctx, RTTDDFT_ERR_UNSUPPORTED, "the adjoint of the Hartree feedback (a state-dependent potential) is not built");
        if (nsteps < 1 || !a_samples || !gdir || !grad || ckpt_every < 1)
            fail(ctx, RTTDDFT_ERR_ARG, "bad argument to rttddft_adjoint");
        if (ctx->opt.propagator != RTTDDFT_PROP_CHEBYSHEV)
            fail(ctx, RTTDDFT_ERR_UNSUPPORTED, "the adjoint differentiates the Chebyshev propagator only");
        if (dv_scale && !ctx->dv_set) fail(ctx, RTTDDFT_ERR_ARG, "dv_scale given before rttddft_set_dv");
        if (dv_scale && ctx->opt.hartree)
            fail(ctx, RTTDDFT_ERR_ARG, "dv_scale is not taken with the Hartree feedback (the density sets the change)");
        sync_and_check(ctx);
        const int nk = ctx->nk, ns = ctx->ns, naux = ctx->naux;
        const size_t vs = (size_t)naux * ns;
        cudaStream_t st = ctx->stream;
        // samples on the host (needed for the gradient formula) and on the device
        const size_t na = 3 * (size_t)nsteps;
        std::vector<double> ha(na), hs;
        if (is_device_ptr(a_samples)) CK(cudaMemcpy(ha.data(), a_samples, na * sizeof(double), cudaMemcpyDeviceToHost));
        else memcpy(ha.data(), a_samples, na * sizeof(double));
        if (!finite_all(ha.data(), na)) fail(ctx, RTTDDFT_ERR_NONFINITE, "a_samples not finite");
        if (dv_scale) {
            hs.resize(nsteps);
            if (is_device_ptr(dv_scale)) CK(cudaMemcpy(hs.data(), dv_scale, nsteps * sizeof(double), cudaMemcpyDeviceToHost));
            else memcpy(hs.data(), dv_scale, nsteps * sizeof(double));
        }
        double a_need = 0.0, s_need = 0.0;
        for (size_t q = 0; q < na; q += 3)
            a_need = std::max(a_need, sqrt(ha[q] * ha[q] + ha[q + 1] * ha[q + 1] + ha[q + 2] * ha[q + 2]));
        for (double x : hs) s_need = std::max(s_need, fabs(x));
        ensure_interval(ctx, std::max(a_need, ctx->opt.a_max), std::max(s_need, ctx->opt.s_max));
        ensure_call_cap(ctx, nsteps);
        CK(cudaMemcpy(ctx->d_a, ha.data(), na * sizeof(double), cudaMemcpyHostToDevice));
        if (dv_scale) CK(cudaMemcpy(ctx->d_dvs, hs.data(), nsteps * sizeof(double), cudaMemcpyHostToDevice));
        // save the state the call must leave unchanged
        CK(cudaMemcpy(&saved, ctx->d_st, sizeof(DevState), cudaMemcpyDeviceToHost));
        for (int k = 0; k < nk; ++k) {
            zd* b = dalloc<zd>(ctx, vs);
            tmp.push_back(b);
            theta_saved.push_back(b);
            CK(cudaMemcpy(b, ctx->hkd[k].theta, vs * sizeof(zd), cudaMemcpyDeviceToDevice));
        }
        restore = true;
        const int N = ctx->nterms;
        const int K = ckpt_every;
        const int nseg = (nsteps + K - 1) / K;
        auto alloc = [&](size_t n) {
            zd* p = dalloc<zd>(ctx, n);
            tmp.push_back(p);
            return p;
        };
        zd* ckpt = alloc((size_t)nseg * nk * vs);   // theta at the start of every segment
        zd* hist = alloc((size_t)(K + 1) * nk * vs);  // theta over the current segment
        zd* Yh = alloc((size_t)nk * N * vs);
        zd* Yb = alloc((size_t)nk * N * vs);
        zd* lam = alloc((size_t)nk * vs);
        const int gblk = std::max(1, std::min(64, (naux * naux + 255) / 256));
        double* gpart = dalloc<double>(ctx, (size_t)nk * gblk * 4);
        tmp.push_back(gpart);
        double* nrm = dalloc<double>(ctx, (size_t)nk * naux);
        tmp.push_back(nrm);
        const int dv_on = dv_scale ? 1 : 0;
        StepArgs a = make_args(ctx, dv_on);
        a.coop_grid = 0;
        StepPlan p = make_plan(ctx);
        auto copy_theta = [&](zd* dst /* nk * vs */, bool to_theta) {
            for (int k = 0; k < nk; ++k) {
                if (to_theta) CK(cudaMemcpyAsync(ctx->hkd[k].theta, dst + (size_t)k * vs, vs * sizeof(zd), cudaMemcpyDeviceToDevice, st));
                else CK(cudaMemcpyAsync(dst + (size_t)k * vs, ctx->hkd[k].theta, vs * sizeof(zd), cudaMemcpyDeviceToDevice, st));
            }
        };
        const double om = ctx->omega, dt = ctx->opt.dt, c = ctx->c;
        // current of the propagated theta at t_m (host sum of the row partials)
        std::vector<double> post((size_t)nk * naux * POST_STRIDE), wk(nk);
        CK(cudaMemcpy(wk.data(), ctx->d_wk, nk * sizeof(double), cudaMemcpyDeviceToHost));
        auto current = [&](double out[3]) {
            launch_subspace_j(a, st);
            KCHECK();
            CK(cudaMemcpyAsync(post.data(), ctx->d_part_post, post.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            for (int l = 0; l < 3; ++l) {
                double v = 0.0;
                for (int k = 0; k < nk; ++k)
                    for (int i = 0; i < naux; ++i) v += wk[k] * post[((size_t)k * naux + i) * POST_STRIDE + 1 + l];
                out[l] = -v / om;
            }
        };
        // ---- forward pass: checkpoints and the dipole increment
        double dmu[3] = {0, 0, 0}, jprev[3] = {saved.jind_prev[0], saved.jind_prev[1], saved.jind_prev[2]};
        for (int m = 0; m < nsteps; ++m) {
            if (m % K == 0) copy_theta(ckpt + (size_t)(m / K) * nk * vs, false);
            // the current uses the sample of the step just taken
            launch_propagate_only(a, p, m, st);
            KCHECK();
            double J[3];
            current(J);
            for (int l = 0; l < 3; ++l) {
                const double jind = J[l] - saved.j_gs[l];
                dmu[l] += om * dt * 0.5 * (jprev[l] + jind);
                jprev[l] = jind;
            }
        }
        if (dmu_out)
            for (int l = 0; l < 3; ++l) dmu_out[l] = dmu[l];
        // ---- reverse sweep, segment by segment
        for (size_t q = 0; q < na; ++q) grad[q] = 0.0;
        launch_zero(lam, (size_t)nk * vs, st);
        std::vector<double> hg((size_t)nk * gblk * 4), hn((size_t)nk * naux), lamh(2 * nk);
        std::vector<double> lamc(LAM_N * nk);
        CK(cudaMemcpy(lamc.data(), ctx->d_lam, lamc.size() * sizeof(double), cudaMemcpyDeviceToHost));
        for (int sg = nseg - 1; sg >= 0; --sg) {
            const int s0 = sg * K, s1 = std::min(nsteps, s0 + K);
            copy_theta(ckpt + (size_t)sg * nk * vs, true);
            copy_theta(hist, false);
            for (int m = s0; m < s1; ++m) {
                launch_propagate_only(a, p, m, st);
                copy_theta(hist + (size_t)(m - s0 + 1) * nk * vs, false);
            }
            KCHECK();
            for (int m = s1; m > s0; --m) {
                const double* am = ha.data() + 3 * (size_t)(m - 1);
                // source from J(t_m): weight of t_m in the trapezoid sum of dmu
                const double wm = om * dt * (m == nsteps ? 0.5 : 1.0);
                const double sm = (gdir[0] * am[0] + gdir[1] * am[1] + gdir[2] * am[2]) / c;
                launch_adj_jterm(a, lam, hist + (size_t)(m - s0) * nk * vs, gdir, sm, -2.0 * wm / om, nrm, st);
                KCHECK();
                CK(cudaMemcpyAsync(hn.data(), nrm, hn.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
                // propagator of step m-1: recompute the Chebyshev vectors from theta_{m-1}
                launch_hsub_only(a, p, m - 1, st);
                for (int k = 0; k < nk; ++k)
                    CK(cudaMemcpyAsync(Yh + (size_t)k * N * vs, hist + (size_t)(m - 1 - s0) * nk * vs + (size_t)k * vs,
                                       vs * sizeof(zd), cudaMemcpyDeviceToDevice, st));
                for (int t = 1; t < N; ++t) launch_adj_fwd_term(a, Yh, N, t, st);
                launch_adj_bwd_init(a, Yb, lam, N, st);
                for (int t = N - 1; t >= 1; --t) launch_adj_bwd_term(a, Yb, N, t, st);
                launch_adj_grad(a, Yh, Yb, N, gpart, gblk, st);
                KCHECK();
                CK(cudaMemcpyAsync(hg.data(), gpart, hg.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
                // lam_{m-1} = theta-bar = ybar_0
                for (int k = 0; k < nk; ++k)
                    CK(cudaMemcpyAsync(lam + (size_t)k * vs, Yb + (size_t)k * N * vs, vs * sizeof(zd),
                                       cudaMemcpyDeviceToDevice, st));
                CK(cudaStreamSynchronize(st));
                double nm = 0.0;
                for (double x : hn) nm += x;
                for (int l = 0; l < 3; ++l) grad[3 * (size_t)(m - 1) + l] += wm * gdir[l] * (-1.0 / om) * nm / c;
                for (int k = 0; k < nk; ++k) {
                    double acc[4] = {0, 0, 0, 0};
                    for (int b = 0; b < gblk; ++b)
                        for (int q = 0; q < 4; ++q) acc[q] += hg[((size_t)k * gblk + b) * 4 + q];
                    const double ilh = lamc[LAM_N * k + 2];
                    for (int l = 0; l < 3; ++l)
                        grad[3 * (size_t)(m - 1) + l] += ilh * (acc[l] / c + am[l] / (c * c) * acc[3]);
                }
            }
        }
        // ---- restore
        for (int k = 0; k < nk; ++k)
            CK(cudaMemcpy(ctx->hkd[k].theta, theta_saved[k], vs * sizeof(zd), cudaMemcpyDeviceToDevice));
        CK(cudaMemcpy(ctx->d_st, &saved, sizeof(DevState), cudaMemcpyHostToDevice));
        restore = false;
        for (void* q : tmp) dfree(ctx, q);
        return RTTDDFT_OK;
    } catch (Fail& f) {
        if (restore) {
            for (size_t k = 0; k < theta_saved.size(); ++k)
                cudaMemcpy(ctx->hkd[k].theta, theta_saved[k], (size_t)ctx->naux * ctx->ns * sizeof(zd),
                           cudaMemcpyDeviceToDevice);
            cudaMemcpy(ctx->d_st, &saved, sizeof(DevState), cudaMemcpyHostToDevice);
        }
        for (void* q : tmp) dfree(ctx, q);
        return f.code;
    }
}

}  // extern "C"

// ------------------------------------------------------------ operator apply without allocation
// Some callers cannot call cudaMalloc at the moment they need the operator:
// code running while a CUDA graph is being captured, allocator-free
// real-time or callback threads, or processes whose device memory is owned
// by another pool.  rttddft_apply_noalloc serves them: its scratch (the
// staged input block, Q = A X, the muffin-tin products, the split-K partials
// and the small descriptors) comes from one file-scope device array that
// every GPU loading this library holds until the process exits.  The caller
// passes device input and output buffers.
#define RTD_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)  // 16 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[RTD_NOALLOC_SCRATCH_BYTES];

#include <mutex>
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[256];  // device address of the array, per device ordinal

// Small host structs reach the scratch array as kernel parameters (no
// staging copy from pageable memory).
struct Blob512 {
    unsigned char b[512];
};
__global__ void k_put_blob(unsigned char* dst, Blob512 src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src.b[i];
}
template <typename T>
static void put_struct(unsigned char* dst, const T& v, cudaStream_t s) {
    static_assert(sizeof(T) <= sizeof(Blob512), "struct too large for a blob");
    Blob512 b;
    memset(&b, 0, sizeof(b));
    memcpy(b.b, &v, sizeof(T));
    k_put_blob<<<1, 128, 0, s>>>(dst, b, (int)sizeof(T));
}

// Resolve the array's device address on the context's device (first call on
// each device; later calls reuse it).  The address is looked up with that
// device current, so the caller's current device must be the context's.
static unsigned char* noalloc_base(rttddft_ctx* ctx) {
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != ctx->device)
        fail(ctx, RTTDDFT_ERR_ARG, "rttddft_apply_noalloc: the current device (" + std::to_string(dev) +
                                       ") is not the context's device (" + std::to_string(ctx->device) + ")");
    if (dev < 0 || dev >= 256) fail(ctx, RTTDDFT_ERR_UNSUPPORTED, "device ordinal above 255");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            fail(ctx, RTTDDFT_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    return (unsigned char*)g_noalloc_addr[dev];
}

extern "C" int rttddft_apply_noalloc(rttddft_ctx* ctx, int k, int ncols, const double* x, const double* a_vec,
                                     double dv_scale, double* hx, double* sx) {
    if (!ctx) return RTTDDFT_ERR_ARG;
    try {
        if (k < 0 || k >= ctx->nk || ncols < 1 || !x || !a_vec || !hx || !sx)
            fail(ctx, RTTDDFT_ERR_ARG, "bad argument to rttddft_apply_noalloc");
        if (dv_scale != 0.0 && !ctx->dv_set) fail(ctx, RTTDDFT_ERR_ARG, "dv_scale != 0 before rttddft_set_dv");
        if (dv_scale != 0.0 && ctx->opt.hartree)
            fail(ctx, RTTDDFT_ERR_UNSUPPORTED, "rttddft_apply_noalloc has no Hartree potential (use rttddft_apply)");
        if (!is_device_ptr(x) || !is_device_ptr(hx) || !is_device_ptr(sx))
            fail(ctx, RTTDDFT_ERR_ARG, "rttddft_apply_noalloc takes device pointers for x, hx and sx");
        if (ctx->toep_global)
            fail(ctx, RTTDDFT_ERR_ARG, "rttddft_apply_noalloc: the table window of this G set does not fit in "
                                       "shared memory (use rttddft_apply)");
        const KDev& K = ctx->hkd[k];
        const int ns = ctx->ns, nb = K.nb, ma = std::max(ctx->at.ma, 1), ng = K.ng;
        const int dv_on = (dv_scale != 0.0) ? 1 : 0;
        const bool f32 = ctx->opt.precision != RTTDDFT_PREC_FP64;
        const int splits = (ng + ctx->kc_fwd - 1) / ctx->kc_fwd;
        // carve the scratch array
        size_t off = 0;
        auto take = [&](size_t bytes) {
            off = (off + 255) & ~(size_t)255;
            const size_t at = off;
            off += std::max(bytes, (size_t)1);
            return at;
        };
        const size_t o_kd = take(sizeof(KDev)), o_gd = take(sizeof(GemmDesc)), o_st = take(sizeof(DevState));
        const size_t o_c = take((size_t)nb * ns * sizeof(zd)), o_y = take((size_t)nb * 2 * ns * sizeof(zd));
        const size_t o_q = take((size_t)ma * ns * sizeof(zd)), o_z = take((size_t)ma * 2 * ns * sizeof(zd));
        const size_t o_part = take((size_t)splits * ns * ma * sizeof(zd));
        const size_t o_jmt = take((size_t)std::max(ctx->at.lrows, 1) * 5 * sizeof(double));
        const size_t o_pf = take((size_t)ctx->max_nback * 5 * sizeof(double));
        const size_t o_pt = take((size_t)ctx->nslot * 2 * ctx->ntsel * ctx->maxng * sizeof(zd));
        const size_t o_vs = dv_on ? take((size_t)ctx->nvt * sizeof(zd)) : 0;
        const size_t o_vs32 = (dv_on && f32) ? take((size_t)ctx->nvt * sizeof(zf)) : 0;
        if (off > RTD_NOALLOC_SCRATCH_BYTES)
            fail(ctx, RTTDDFT_ERR_ARG, "rttddft_apply_noalloc needs " + std::to_string(off) +
                                           " bytes of scratch for this k-point; the static limit is " +
                                           std::to_string(RTD_NOALLOC_SCRATCH_BYTES) + " bytes");
        unsigned char* base = noalloc_base(ctx);
        cudaStream_t st = ctx->stream;
        KDev kc = K;
        kc.C = (zd*)(base + o_c);
        kc.Y = (zd*)(base + o_y);
        kc.Q = (zd*)(base + o_q);
        kc.Z = (zd*)(base + o_z);
        GemmDesc g{};
        g.A = f32 ? (const void*)K.at32 : (const void*)K.at;
        g.B = kc.C;
        g.C = kc.Q;
        g.M = ctx->at.ma;
        g.K = ng;
        g.lda = ng;
        g.ldb = nb;
        g.ldc = ma;
        g.part_off = 0;
        DevState ds{};
        for (int l = 0; l < 3; ++l) ds.cur_a[l] = a_vec[l];
        ds.cur_s = dv_scale;
        ds.cur_aa = (a_vec[0] * a_vec[0] + a_vec[1] * a_vec[1] + a_vec[2] * a_vec[2]) / (2 * ctx->c * ctx->c);
        put_struct(base + o_kd, kc, st);
        put_struct(base + o_gd, g, st);
        put_struct(base + o_st, ds, st);
        KCHECK();
        StepArgs a = make_args(ctx, dv_on);
        a.kd = (const KDev*)(base + o_kd);
        if (a.prec >= 2) a.prec = 1;  // the static scratch holds the FP32-form operands only
        a.vsteps = nullptr;
        a.tcback = 0;
        a.ith = 0;  // the interstitial sum from the table (the FFT buffers belong to the context)
        a.nk = 1;
        a.st = (DevState*)(base + o_st);
        a.part_jmt = (double*)(base + o_jmt);
        a.part_full = (double*)(base + o_pf);
        a.part_t = (zd*)(base + o_pt);
        a.mtg = nullptr;  // the muffin-tin GEMM buffers belong to the context: per-row kernel instead
        a.mtw = nullptr;
        if (dv_on) {
            a.vstep = (zd*)(base + o_vs);
            a.vstep32 = f32 ? (zf*)(base + o_vs32) : nullptr;
        }
        StepPlan p = make_plan(ctx);
        p.fft = nullptr;
        p.side = nullptr;
        p.tile_cnt = nullptr;  // the context's counters may be in use on another stream
        p.gd_mt1 = nullptr;
        p.gd_fwd = (const GemmDesc*)(base + o_gd);
        p.maxng = ng;
        p.part = (zd*)(base + o_part);
        if (dv_on) launch_vstep(a, st);
        const zd* xz = (const zd*)x;
        zd* hz = (zd*)hx;
        zd* sz = (zd*)sx;
        for (int c0 = 0; c0 < ncols; c0 += ns) {
            const int w = std::min(ns, ncols - c0);
            if (w < ns) launch_zero(kc.C, (size_t)nb * ns, st);  // unused columns start at zero
            CK(cudaMemcpyAsync(kc.C, xz + (size_t)c0 * nb, (size_t)w * nb * sizeof(zd), cudaMemcpyDeviceToDevice, st));
            launch_operator_pass(a, p, st);
            KCHECK();
            CK(cudaMemcpyAsync(hz + (size_t)c0 * nb, kc.Y, (size_t)w * nb * sizeof(zd), cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(sz + (size_t)c0 * nb, kc.Y + (size_t)ns * nb, (size_t)w * nb * sizeof(zd),
                               cudaMemcpyDeviceToDevice, st));
        }
        return RTTDDFT_OK;
    } catch (Fail& f) {
        return f.code;
    }
}

extern "C" int rttddft_zgemm_bf16x3(int trans, int m, int n, int k, const double* a, int lda, const double* x,
                                    int ldx, double* c, int ldc, int beta_add, void* stream) {
    if (m < 0 || n < 0 || k < 0 || (trans != 0 && trans != 1)) return RTTDDFT_ERR_ARG;
    if (m == 0 || n == 0) return RTTDDFT_OK;
    if (!a || !x || !c) return RTTDDFT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (k == 0) {
        if (!beta_add) {
            if (ldc < m) return RTTDDFT_ERR_ARG;
            if (cudaMemset2DAsync(c, (size_t)ldc * 16, 0, (size_t)m * 16, n, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return RTTDDFT_ERR_CUDA;
        }
        return RTTDDFT_OK;
    }
    if (!is_device_ptr(a) || !is_device_ptr(x) || !is_device_ptr(c)) return RTTDDFT_ERR_ARG;
    return tc_zgemm(trans, m, n, k, (const zd*)a, lda, (const zd*)x, ldx, (zd*)c, ldc, beta_add, s);
}
