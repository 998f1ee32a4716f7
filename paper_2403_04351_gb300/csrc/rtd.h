// Internal layout of the rttddft device state and the kernel launchers.
#pragma once
#include <string>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "common.cuh"

#define RTD_MAX_ATOMS 64
#define RTD_MAX_TERMS 512
#define RTD_REC_STRIDE 16  // doubles per step record
#define BT 128            // plane-wave rows (and G' columns) per tile of the slot kernels
#define BKB 32            // plane-wave rows per block of the [HC | SC] row kernel k_back
#define LAM_N 8           // doubles per k-point of the Chebyshev scaling record

// Record fields (offsets within one record)
enum { REC_T = 0, REC_J = 1, REC_JF = 4, REC_DMU = 7, REC_E = 10, REC_NDEV = 11,
       REC_RES = 12, REC_DTCR = 13, REC_NEXC = 14 };

// One entry of a batched GEMM; batched kernels index an array of these
// with blockIdx.z.  Matrices are complex column-major.
struct GemmDesc {
    const void* A;   // zd or zf
    const zd* B;
    zd* C;
    int M, K;        // output rows, contraction length
    int lda, ldb, ldc;
    size_t part_off; // offset (complex elements) of this entry's split-K partials
};

// Batched Toeplitz entry: Y[G, n] (+)= sum_G' tab(G - G') X[G', n] + d_G X[G, n]
struct ToepDesc {
    const zd* X;
    zd* Y;
    int ldx, ldy;
};

// Per-atom tables
struct AtomTab {
    int n;                       // atoms
    int na[RTD_MAX_ATOMS];       // matching rows N_A
    int nlo[RTD_MAX_ATOMS];      // local orbitals
    int m[RTD_MAX_ATOMS];        // na + nlo
    int aoff[RTD_MAX_ATOMS];     // first row in A / Q / Z
    int looff[RTD_MAX_ATOMS];    // first LO (relative to N_G)
    int loff[RTD_MAX_ATOMS];     // first row of the atom in stacked local blocks
    size_t boff[RTD_MAX_ATOMS];  // offset (complex) of the atom's m x m block
    int lrows;                   // sum m
    int ma;                      // sum na
    int nlo_tot;                 // sum nlo
};

// Per-k device pointers (an array of these lives in device memory)
struct KDev {
    int ng, nb;
    zd* caux;     // nb x naux
    zf* caux32;   // nb x naux (FP32 form)
    zd* at;       // ng x ma: A^H, the matching coefficients conjugate-transposed
    zf* at32;     // ng x ma (FP32 form)
    int* glin;    // ng  linear table index of G
    double* gk;   // ng x 3 (row-major)
    double* eps;  // naux
    zd* psub;     // 3 x naux x naux
    zd* lloc;     // lrows x naux: local coordinates [A_a CC_G ; CC_l] of the aux basis
    zd* theta;    // naux x ns
    zd* theta_t;  // naux x ns  CC^H S C
    zd* ring;     // 3 x naux x ns  Chebyshev vectors
    zd* acc;      // naux x ns
    zd* hsub;     // naux x naux
    zd* dvsub;    // naux x naux  (potential change, when active)
    zd* C;        // nb x ns
    zd* Y;        // nb x 2ns  [H C | S C]
    zd* Q;        // ma x ns
    zd* Z;        // ma x 2ns
    zd* th;       // ng x ns  interstitial convolution V~ * C_G (tensor-core form)
    zd* tb;       // ng x 2ns back-projection A^H [hQ | oQ] (tensor-core form)
    zd* gram;     // ns x ns x 2   theta^H theta~ and theta~^H theta~
    zd* evec;     // naux x naux (EIG form)
    double* eval; // naux
    zd* wtmp;     // naux x ns
    zd* coef;     // RTD_MAX_TERMS Chebyshev coefficients
    double* lam;  // [LAM_N]: centre, half-width, 1/half-width, cos and sin of -dt*centre
    double dtcr_b;// dt_cr from the bounds of the call
    double pad;
};

// Device-resident step state
struct DevState {
    int cstep;          // step index within the current rttddft_step call
    int rec_count;
    long long gstep;    // steps since set-up
    double t;           // time of the current state
    double dmu[3];
    double jind_prev[3];
    double j_gs[3];
    double cur_a[3];    // A of the current step
    double cur_s;       // potential-change scale of the current step
    double cur_aa;      // |A|^2 / (2 c^2)
    int err;            // nonzero: a device iteration limit ran out
    unsigned bar;       // arrival counter of the grid barrier (zeroed by k_hsub and k_finalize)
};

// Everything the step kernels need, passed by value
struct StepArgs {
    int nk, ns, naux, prop, prec, reproject, nterms, dv_on;
    int vt_center, nvt, lrows, ma, rec_cap, pad;
    double dt, c, omega;
    double inv_c, half_inv_c2;  // 1/c and 1/(2 c^2): GB300 FP64 division is slow, multiply instead
    const KDev* kd;
    const double* occ;   // ns
    const double* wk;    // nk
    const zd* h;         // atom blocks (boff)
    const zd* o;         // atom blocks (boff)
    const zd* p;         // 3 blocks per atom at 3*boff
    const zf* h32;       // FP32 copies of h, o, p (FP32 and split-BF16 forms)
    const zf* o32;
    const zf* p32;
    const zd* dh;        // potential change blocks (or null)
    const zd* vtab;      // V~
    const zf* vtab32;
    const zd* dvtab;     // dV~ (or null)
    zd* vstep;           // per-step combined table V~ + s dV~
    zf* vstep32;
    const uint2* vtabs;  // V~ split for the tensor cores: (Re hi | Re lo << 16, Im hi | Im lo << 16)
    uint2* vsteps;       // the same for the per-step table
    const double* a;     // call samples [cstep][3]
    const double* dvs;   // call dv scales (or null)
    DevState* st;
    double* rec;         // records
    double* part_jmt;    // [nk][lrows][5]  per local row: J_mt (3), LO-row E and c^H S c
    double* part_full;   // [nk][max_nback][5] per back tile: E, c^H S c, sum (G+k)|c|^2 (3)
    double* part_post;   // [nk][naux][POST_STRIDE]  per subspace row
    const AtomTab* at;   // device copy
    const GemmDesc* gd_proj;  // projection descriptors (split-K partial offsets)
    const zd* part_proj;      // projection split-K partials
    int kc_proj, max_nback;
    int wmax;                 // largest table window of a back tile (entries)
    int nseg, segw, maxng;    // G' segments of the interstitial sum
    int msegw, nslot;         // matching rows per back-projection slot; nseg + such slots
    zd* part_t;               // [nk][nslot][2 NT][maxng] slot partial sums
    int* flag;                // device error flags (bit 0 Jacobi, 1 bounds, 2 barrier)
    int coop_grid;            // blocks of the cooperative Chebyshev launch (0: per-term launches)
    int kofs;                 // k-point of kd[0] (single-k operator calls), 0 in the step
    int tcback;               // the back-projection runs on the tensor cores (split-BF16 form)
    int at_n, at_maxm;        // atoms, and the largest local block m = N_A + n_lo
    int tc_fmt;               // tensor-core operand format: 1 bf16, 0 fp16
    int ith;                  // the interstitial sum arrives in K.th (tensor cores or FFT)
    int hartree;              // the potential change is the Hartree potential of the density (FFT route)
    int cheb_tile;            // the cooperative series runs as k_cheb_tile (4 < N_s <= 64)
    double tc_st;             // scale of the split table (fp16 range)
    double mt_u;              // muffin-tin part of the density feedback: dh = mt_u (n - n0) (0: off)
    const zd* mtn0;           //   reference muffin-tin density matrices n_a(0) (atom blocks at boff)
    zd* mty;                  //   per k the local coordinates L theta of the state (lrows x ns)
    const double* mt_lnorm;   //   per atom max_k ||L_ka||_F^2 (the bound's factor)
    double* mt_fn2;           //   per atom ||dh_a||_F^2 of the step (accumulated, reset by k_mt_bound)
    zf* dh32;                 //   FP32 copy of dh (reduced-precision rebuild)
    double* part_fin;         // [nk][FIN_CH][FIN_STRIDE] first-phase sums of the step's reductions
    double* gdev;             // [nk][ns] largest |C^H S C - I| per column (many states)
    int toep_global;          // the direct sum gathers the table through L1/L2 into K.th (window too large)
    zf* mtg;                  // muffin-tin products as GEMMs: per atom the 5m x m stack [h_eff; o; p_x; p_y; p_z]
    zd* mtw;                  //   per (k, atom) its product with [Q; C_lo] (5m x N_s, stride mtw_stride)
    zd* mtv;                  //   per (k, atom) the gathered [Q; C_lo] (m x N_s, stride mtv_stride)
    int mtw_stride, mtv_stride;
};
#define ZT_MIN_N 16           // columns from which the FP32 contractions take the 64 x 64 tiled kernel
#define JRHO_MIN_NS 8         // above this many states the subspace current goes through rho = theta F theta^H
#define FIN_CH 8              // row chunks per k-point of the first reduction phase
#define FIN_STRIDE 16
#define POST_STRIDE 36        // part_post row: residual, J_sub (3), then theta^H theta~ (ns <= 4)

// ---- k_linalg.cu
void launch_gemm_nn(const GemmDesc* d, int nbatch, int maxM, int maxK, int N, int kchunk,
                    zd* part, int beta_add, bool a_fp32, const double* dscale, cudaStream_t s);
// returns true when the split-K slices were also summed into C by the launch
// itself (FP32 streaming kernel with tile counters: the last slice of a row
// tile sums them in slice order); otherwise a split launch needs
// launch_split_reduce.  tile_cnt: zeroed, one counter per (row tile, batch).
bool launch_gemm_cn(const GemmDesc* d, int nbatch, int maxM, int maxK, int N, int kchunk,
                    zd* part, int beta_add, bool a_fp32, const double* dscale, cudaStream_t s,
                    unsigned* tile_cnt = nullptr);
void launch_split_reduce(const GemmDesc* d, int nbatch, int maxM, int N, int kchunk, const zd* part,
                         int beta_add, cudaStream_t s);
// dmode: 0 none, 1 kinetic |G+k|^2/2, 2..4 (G+k)_{x,y,z}, 5 unit
void launch_toeplitz(const KDev* kd, const ToepDesc* td, int nk, int maxng, int N, const zd* tab,
                     int center, int beta_add, int dmode, const double* dscale, cudaStream_t s);
void launch_zero(zd* p, size_t n, cudaStream_t s);
void launch_copy_rows(const GemmDesc* d, int nbatch, int maxrows, int ncol, cudaStream_t s);
void launch_convert_f32(const zd* src, zf* dst, size_t n, cudaStream_t s);
// AT (n x m) = A^H for A (m x n), both column-major
void launch_conj_transpose(const zd* A, zd* AT, int m, int n, cudaStream_t s);

// ---- k_step.cu
struct StepPlan {
    int maxnb, maxng, nterms;
    const GemmDesc *gd_expand, *gd_fwd, *gd_proj, *gd_g1, *gd_g2, *gd_evh, *gd_evn;
    zd* part;
    int kc_fwd, kc_proj, kc_expand;
    // potential change (a2)
    const GemmDesc *gd_dvw, *gd_dvg, *gd_dvi;   // W = dh L, dV = L^H W, dV += C_G^H T
    const GemmDesc* gd_dvi32;                    // dV += C_G^H T with FP32 C_G (tensor-core forms)
    const GemmDesc *gd_dvw32, *gd_dvg32;         // W = dh L, dV = L^H W from FP32 dh and L (or null)
    zd* part_dv;                                 // its split-K partials
    int kc_dvi;
    const ToepDesc* td_dv;                       // T = dV~ C_G
    int n_dvw;                                   // entries of gd_dvw (nk * atoms)
    int maxm;
    int* d_flag;
    zd* const* jac_mats; double* const* jac_vals; zd* const* jac_vecs;
    int max_sweeps;
    const struct TcPlan* tc;  // tensor-core operator plan (split-BF16 form) or null
    const struct TcCC* tcc;   // tensor-core expansion and projection (split forms, many states) or null
    const struct TcMT* tcmt;  // tensor-core muffin-tin blocks (split-BF16 form, many states) or null
    const struct FftPlan* fft;  // FFT route of the interstitial convolution or null
    unsigned* tile_cnt;         // zeroed row-tile counters of the fused split-K sums (or null)
    cudaStream_t side;          // second stream for work that overlaps the main chain (or null)
    int fft_launches;           // launches of one FFT convolution (3 or 5)
    const GemmDesc* gd_exp64;   // Hartree feedback in the FP32 form: C in FP64 for the density (or null)
    const ToepDesc* td_dens;    // per k: the C the density is taken from
    cudaEvent_t ev_fork, ev_join;
    const ToepDesc* td_op;      // per k: {C, th}: the operator's convolution source and destination
    const GemmDesc* gd_mt1;     // per (k, atom): [h_eff; o; p] times the gathered [Q; C_lo] (or null)
    const GemmDesc* gd_mty;     // per k: L theta, the state's local coordinates (muffin-tin feedback) or null
};
// Optional per-kernel tracing: an event is recorded after every launch of a step.
struct TraceHook {
    cudaEvent_t* ev;     // capacity events
    const char** names;  // name of the kernel that ends at ev[i]
    int n, cap;
};
void launch_step(const StepArgs& a, const StepPlan& p, cudaStream_t s, int* nlaunch,
                 TraceHook* tr = nullptr);
int launch_operator_pass(const StepArgs& a, const StepPlan& p, cudaStream_t s, TraceHook* tr = nullptr);
int prepare_back_kernels(const StepArgs& a);
// blocks for the cooperative Chebyshev launch if it can be captured in a graph, else 0
// tile: set to 1 when the series for many states runs in tiles of HH rows (k_cheb_tile)
int prepare_cheb_coop(const StepArgs& a, cudaStream_t s, int* tile);
void launch_cheb_coop(const StepArgs& a, cudaStream_t s);
void launch_prep_coef(const StepArgs& a, cudaStream_t s);
void launch_subspace_current(const StepArgs& a, int set_gs, cudaStream_t s);
void launch_set_cur(const StepArgs& a, cudaStream_t s);
void launch_vstep(const StepArgs& a, cudaStream_t s);
void launch_check_samples(const double* a, int na, double amax, const double* s, int ns, double smax,
                          int* flag, cudaStream_t st);
int launch_jacobi(zd* const* mats, double* const* vals, zd* const* vecs, int nbatch, int n,
                  int max_sweeps, int* d_flag, cudaStream_t s);
void launch_phase_fix(const KDev* kd, int nk, int naux, zd* const* extra, const int* ldextra,
                      int nextra_rows, cudaStream_t s);
void launch_scale_cols(zd* const* mats, const double* const* vals, int nbatch, int n, int mode,
                       cudaStream_t s);

// ---- adjoint (k_step.cu, k_adjoint.cu)
void launch_propagate_only(const StepArgs& a, const StepPlan& p, int cstep, cudaStream_t s);
void launch_hsub_only(const StepArgs& a, const StepPlan& p, int cstep, cudaStream_t s);
void launch_subspace_j(const StepArgs& a, cudaStream_t s);
// muffin-tin density matrices of theta: the reference n0 (set-up) or dh = U (n - n0) and its bound term
int launch_mt_feedback(const StepArgs& a, const StepPlan& p, int reference, double* l1, cudaStream_t s);
void launch_mt_lnorm(const StepArgs& a, cudaStream_t s);
void launch_adj_fwd_term(const StepArgs& a, zd* Yh, int nterm, int nt, cudaStream_t s);
void launch_adj_bwd_init(const StepArgs& a, zd* Yb, const zd* lam, int nterm, cudaStream_t s);
void launch_adj_bwd_term(const StepArgs& a, zd* Yb, int nterm, int nt, cudaStream_t s);
void launch_adj_grad(const StepArgs& a, const zd* Yh, const zd* Yb, int nterm, double* part, int nblk,
                     cudaStream_t s);
void launch_adj_jterm(const StepArgs& a, zd* lam, const zd* theta, const double* g, double sm, double cfac,
                      double* nrm, cudaStream_t s);

// ---- tensor-core split-BF16 operator (k_tc.cu)
struct TcPlan;
// fmt: 1 split-BF16, 0 split-FP16 (operands scaled by powers of two: sa for the
// matching coefficients, st for the table, fixed scales for C and Z)
// interstitial convolution by FFT (k_fft.cu)
struct FftPlan;
int fft_grid_for(const int vt_dim[3], int F[3]);
int fft_plan_create(FftPlan** out, int nk, const int* ng, const int* const* gint, const int vt_dim[3],
                    const zd* vtab_dev, int ncol, int prec, cudaStream_t st, std::string* why);
int fft_set_dv(FftPlan* pl, const zd* dvtab_dev, const int vt_dim[3], int ncol, cudaStream_t st, std::string* why);
void fft_plan_destroy(FftPlan* pl);
void fft_plan_info(const FftPlan* pl, int F[3], int* fused);
int fft_tune(FftPlan* pl, const ToepDesc* td, int ncol, cudaStream_t st);
int fft_reserve_columns(FftPlan* pl, int ncol, cudaStream_t st, std::string* why);
int fft_hartree_init(FftPlan* pl, const double recip[9], const int vt_dim[3], double omega, double bound, int ns,
                     cudaStream_t st, std::string* why);
int launch_fft_density(const FftPlan* pl, const ToepDesc* td, int nk, int ns, const double* occ, const double* wk,
                       int reference, cudaStream_t st);
double* fft_l1(const FftPlan* pl);
int launch_fft_hartree(const FftPlan* pl, const ToepDesc* td, int nk, int ns, const double* occ, const double* wk,
                       int* flag, cudaStream_t st);
int launch_fft_conv(const FftPlan* pl, const ToepDesc* td, int kofs, int nk, int ncol, int vmode, int use_vd,
                    const double* s, cudaStream_t st);

int tc_plan_create(TcPlan** out, int nk, int ns, int ma, const int* ng, const int* const* glin_host,
                   const zd* const* at_dev, const zd* vtab, int nvt, int vt_center, const KDev* d_kd,
                   int fmt, double sa, double st, cudaStream_t s, std::string* why);
double tc_table_scale(const TcPlan* tp);
int tc_format(const TcPlan* tp);
void tc_plan_destroy(TcPlan* tp);
// NT, 100 x generated stages + copied stages, K blocks per slice, slices, window, smem of the
// interstitial launch, candidates tuned, tuned interstitial and matching-row times (ns)
void tc_plan_info(const TcPlan* tp, int* v);
void launch_tc_pack(const TcPlan* tp, const StepArgs& a, cudaStream_t s);
int launch_tc_operator(const TcPlan* tp, const StepArgs& a, cudaStream_t s, bool rows_only = false);
void launch_tc_reduce(const TcPlan* tp, const StepArgs& a, cudaStream_t s, bool rows_only = false);
bool tc_has_back(const TcPlan* tp);  // the back-projection runs on the tensor cores (4 N_s <= 256)
int tc_dv_prepare(TcPlan* tp, const zd* const* caux_dev, const int* nb, const int* ng, int naux, int nvt,
                  cudaStream_t s, std::string* why);
void tc_dv_set_table(TcPlan* tp, const zd* dvtab, int nvt, double vmax, cudaStream_t s);
bool tc_dv_ready(const TcPlan* tp);
int tc_dv_tiles(const TcPlan* tp);
void launch_tc_dv_toeplitz(const TcPlan* tp, const StepArgs& a, const ToepDesc* td, cudaStream_t s);
int launch_tc_back(const TcPlan* tp, const StepArgs& a, cudaStream_t s);
// expansion and projection with the auxiliary basis on the tensor cores (split-BF16, many states)
struct TcCC;
int tc_cc_create(TcCC** out, int nk, int naux, int ns, const int* nb, const zd* const* cc_dev, int* flag,
                 cudaStream_t s, std::string* why);
void tc_cc_destroy(TcCC* t);
int launch_tcc_expand(const TcCC* t, const StepArgs& a, cudaStream_t s);
int launch_tcc_project(const TcCC* t, const StepArgs& a, zd* part, cudaStream_t s);
// the muffin-tin blocks of every (k, atom) as one batch on the tensor cores (split-BF16, many states)
struct TcMT;
int tc_mt_create(TcMT** out, int nk, int nat, int maxm, int ns, int* flag, cudaStream_t s, std::string* why);
void tc_mt_destroy(TcMT* t);
int launch_tc_mt(const TcMT* t, const StepArgs& a, cudaStream_t s);
// ---- tensor-core split-BF16 complex GEMM (k_tc.cu); returns an RTTDDFT_* code
int tc_zgemm(int opA, int M, int N, int K, const zd* A, int lda, const zd* X, int ldx, zd* C, int ldc,
             int beta_add, cudaStream_t s);
