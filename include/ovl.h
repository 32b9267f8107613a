/*
 * ovl.h -- C ABI of the GB300 (sm_103a) library that approximates
 *          y = sgn(H_w(mu)) b by deflated Arnoldi.
 *
 * Method: Bloch, Wettig, Frommer, Lang, "An iterative method to compute the
 * overlap Dirac operator at nonzero chemical potential" (Lattice 2007,
 * arXiv:0710.0341).
 *
 * Conventions shared by every call
 * --------------------------------
 * Lattice dims[4] = {Lx, Ly, Lz, Lt}; site index n = x + Lx*(y + Ly*(z + Lz*t)).
 * Canonical spinor layout (host or device): complex128 psi[n][spin 4][colour 3]
 *   stored as interleaved doubles (re, im): 24 doubles per site, N = 12 V complex.
 * Canonical link layout: complex128 U[n][nu 0..3 = x,y,z,t][a 3][b 3], 72
 *   doubles per direction and site, 288 per site.
 * Gamma matrices: Hermitian chiral basis with gamma_5 = diag(1, 1, -1, -1)
 *   (the paper says only "Euclidean"; this basis is the library's reading).
 * Pointers: every double/float pointer may be host or device memory; the
 *   library detects which (cudaPointerGetAttributes). Device pointers must
 *   be on the lattice's device. The caller owns every buffer it passes; the
 *   library owns its internal workspace (Krylov bases, deflation vectors,
 *   Newton work) and frees it in the matching destroy call.
 * Streams: work is issued on the stream given to ovl_create_lattice; every
 *   call returns after the result is complete (it synchronises that stream),
 *   so status codes are synchronous.
 * Errors: every call returns 0 (OVL_OK) or one of the codes below and keeps a
 *   message for ovl_last_error(). A failed call leaves its outputs undefined
 *   and the handle usable.
 * Threads: a handle is not thread-safe; use one handle per host thread.
 */
#ifndef OVL_H
#define OVL_H

#ifdef __cplusplus
extern "C" {
#endif

#define OVL_OK        0
#define OVL_EINVAL    1  /* bad argument: sizes, null pointers, mismatched mu/m_w */
#define OVL_ENOMEM    2  /* device allocation failed or over the workspace budget */
#define OVL_ECUDA     3  /* a CUDA runtime call failed */
#define OVL_ENOCONV   4  /* Newton or eigensolver hit its iteration limit */
#define OVL_ETIMEOUT  5  /* a device-side wait gave up after its iteration limit */
#define OVL_ENOTSUP   6  /* combination not supported by this build */

typedef struct ovl_lattice_s*    ovl_lattice;
typedef struct ovl_deflation_s*  ovl_deflation;

/* Arithmetic of the Arnoldi path (ovl_sign_params.prec). */
#define OVL_PREC_FP64       0  /* FP64 stencil; basis stored as FP32 hi+lo pairs (48-bit);
                                  pass-A inner products with FP32 products (they only steer
                                  orthogonality), pass B, projections and recombination in
                                  double-float (48-bit) accumulation, FP64 small-step scalars,
                                  double-float Newton (newton_fp64 = 0) */
#define OVL_PREC_MIXED      1  /* FP32 stencil (18-real links), FP32 basis, FP64 coefficients */
#define OVL_PREC_MIXED_R12  2  /* as OVL_PREC_MIXED with 12-real (two-row) links */
#define OVL_PREC_FP64_DFSTENCIL 3  /* as OVL_PREC_FP64 with the stencil's arithmetic in double-float
                                      (OVL_LINKS_F64DF) on the FP32 pipes */
#define OVL_PREC_FP64_PLAIN 4  /* plain FP64 throughout: FP64 stencil, complex128 basis, FP64
                                  products and sums in both Gram-Schmidt passes, the projections and
                                  the recombination, FP64 Gauss-Jordan Newton (newton_fp64 is
                                  ignored); the reference form the mixed modes are measured against */
#define OVL_PREC_DF40       5  /* as OVL_PREC_FP64 with the Krylov columns' low parts stored as BF16
                                  (FP32 hi + BF16 lo, about 32 significant bits per entry, 12 bytes
                                  per complex entry instead of 16); deflation vectors keep 48 bits */

/* Deflation scheme (Sec. 3 Schur, Sec. 4 LR). */
#define OVL_DEFL_NONE   0
#define OVL_DEFL_SCHUR  1
#define OVL_DEFL_LR     2

/* Packed (internal) spinor formats for the stencil-only entry points. */
#define OVL_VEC_F64  0   /* complex128 */
#define OVL_VEC_F32  1   /* complex64  */
/* Link formats for the stencil-only entry points. */
#define OVL_LINKS_F64    0
#define OVL_LINKS_F32    1
#define OVL_LINKS_R12    2
#define OVL_LINKS_F64DF  3  /* FP64 links and spinors, double-float arithmetic (hi + lo FP32,
                             * about 2^-46 relative error per application) on the FP32 pipes */

typedef struct {
    double mu;          /* chemical potential (Eq. 2) */
    double m_w;         /* Wilson mass, kappa = 1/(8 + 2 m_w), m_w in (-2, 0) */
    int    k;           /* Krylov depth (Eq. 7); 1 <= k */
    int    prec;        /* OVL_PREC_* */
    int    newton_max_iter;  /* <= 0: default 100 */
    double newton_tol;       /* <= 0: default 1e-13 (relative Frobenius step) */
    int    newton_fp64;      /* 0 (default): double-float Gauss-Jordan Newton (one thread-block
                              * cluster per matrix when its rows fit the cluster's shared memory,
                              * else the cooperative kernel), finished by Newton-Schulz steps
                              * once a step is below 3e-2 and |I - X^2|_F < 1/2;
                              * 1: FP64 Gauss-Jordan Newton; 2: double-float Gauss-Jordan Newton,
                              * cooperative kernel only; 3: as 0 without Newton-Schulz;
                              * 4: as 0 with every Newton-Schulz step declined, so that the
                              * iteration returns to Gauss-Jordan (tests that path) */
    /* Adaptive Krylov depth (not in the paper): with adapt_every = d > 0 the
     * solve starts checking at depth k and then every d steps up to k_max:
     * the estimate est_j = |g_j - (g_{j-d}; 0)| / |g_j| compares the
     * small-space coefficient vectors of successive approximations
     * (g = sgn(H) c, the coordinates of y in the orthonormal basis), and the
     * solve stops at the first j with est_j <= tol / 10. */
    int    adapt_every;      /* 0: fixed k */
    int    k_max;            /* upper bound of the adaptive depth (>= k) */
    double tol;              /* target relative error of y (default 1e-8) */
    /* Schur deflation (one value per batch): 0 (default) sgn of the whole
     * (m + k) block matrix of Eq. 15 (Eq. 16, which equals Eq. 19 through
     * Eq. 17); 1 the Sylvester route: sgn(T_m) and sgn(H_k) by the Newton
     * kernels on the two diagonal blocks, the coupling block Y from the
     * Sylvester equation of Eq. 18 (FP64, row by row: T_m is triangular),
     * then Eq. 19. Ignored by LR and undeflated solves. */
    int    schur_route;
} ovl_sign_params;

typedef struct {
    int    status;        /* per-solve OVL_* code */
    int    k_used;        /* Krylov depth reached (< k on an exact invariant subspace) */
    int    m_used;        /* deflated vectors */
    int    newton_iters;  /* scaled Newton iterations for sgn of the small matrix */
    double beta;          /* |x_perp| or |x_minus|: norm of the Krylov start vector */
    double beta_k;        /* H_{k+1,k}, the last Arnoldi residual norm */
    double err_est;       /* last adaptive estimate (0 when k was fixed) */
} ovl_sign_info;

/* ---- lattice and links ------------------------------------------------ */

/* Create a lattice of dims {Lx,Ly,Lz,Lt} (each >= 2) on the current CUDA
 * device. antiperiodic_t != 0 flips the sign of hops across the t boundary
 * (the paper states no boundary condition; periodic is the default).
 * stream: a cudaStream_t (NULL = legacy default stream). */
int ovl_create_lattice(const int dims[4], int antiperiodic_t, void* stream, ovl_lattice* out);
int ovl_destroy_lattice(ovl_lattice lat);

/* Upload SU(3) links U_{n,nu} of Eq. 2 in the canonical layout. Builds the
 * FP64, FP32 and 12-real (rows 0 and 1; row 2 = conj(row0 x row1)) copies. */
int ovl_set_links(ovl_lattice lat, const double* U);

/* ---- the operator (Sec. 1, Eq. 2): y = H_w(mu) x = gamma_5 D_w(mu) x ---- */

/* nrhs right-hand sides, canonical layout, stride 24*V doubles between them.
 * links: OVL_LINKS_* selects the stencil arithmetic (F64: FP64; F64DF: double-float on
 * FP64 data; F32/R12: FP32). */
int ovl_apply_Hw(ovl_lattice lat, double mu, double m_w, const double* in, double* out,
                 int nrhs, int links);

/* ovl_apply_Hw without any device allocation, for callers that cannot let
 * the library allocate (all free HBM handed to the caller's own pool, code
 * that must avoid the implicit synchronisation of cudaMalloc/cudaFree, or a
 * runtime that accounts for every device byte up front). The paper has no
 * counterpart: this is an allocation-free variant of ovl_apply_Hw.
 * in/out: device pointers only (canonical layout, nrhs vectors); results
 * equal ovl_apply_Hw's. Staging uses one fixed 32 MiB device array that every
 * GPU loading the library holds until exit; 2 * nrhs packed spinors plus 24
 * bytes per right-hand side must fit (OVL_EINVAL otherwise). The first call
 * on a device looks up that array's address (cudaGetSymbolAddress). Each call
 * copies a host table and synchronises the lattice's stream, so it may not be
 * made while that stream is being captured (OVL_EINVAL). Calls share the
 * array: calls that overlap on the GPU race. Never calls cudaMalloc or
 * cudaFree. */
int ovl_apply_Hw_noalloc(ovl_lattice lat, double mu, double m_w, const double* in, double* out,
                         int nrhs, int links);

/* Stencil on packed spinors (the library's internal site order), for timing
 * the stencil alone. in/out: device pointers, nrhs vectors of 12*V complex in
 * format fmt (OVL_VEC_*); mu: nrhs chemical potentials (host array).
 * fmt F64 requires links F64 or F64DF; fmt F32 takes F32 or R12 links. */
int ovl_apply_Hw_packed(ovl_lattice lat, const double* mu, double m_w, const void* in,
                        void* out, int nrhs, int fmt, int links);
/* Canonical complex128 <-> packed format (device or host canonical side;
 * packed side must be device memory). */
int ovl_pack_spinor(ovl_lattice lat, const double* canon, void* packed, int nrhs, int fmt);
int ovl_unpack_spinor(ovl_lattice lat, const void* packed, double* canon, int nrhs, int fmt);

/* ---- deflation data (Sec. 3 Eq. 13; Sec. 4 Eq. 20) --------------------- */

/* Import m critical eigenvectors computed elsewhere.
 *  scheme OVL_DEFL_SCHUR: S_or_R = S_m, m orthonormal Schur vectors (m
 *    canonical spinors, one after another); T = T_m, m x m complex128
 *    column-major with A S_m = S_m T_m (upper triangular per Eq. 13; the
 *    Sylvester route, schur_route = 1, needs the triangular form). The
 *    relation is not checked but is used: the update pass of the Arnoldi
 *    step takes A S_m from S_m T_m, so data that miss it by delta give
 *    results off by about delta times the reorthogonalisation coefficients
 *    (1e-7 of |b| for delta of order one). T may be non-diagonalisable (the
 *    small sign never forms eigenvectors). L must be NULL.
 *  scheme OVL_DEFL_LR: S_or_R = R_m right eigenvectors, T = Lambda_m (m
 *    complex128 eigenvalues), L = L_m left eigenvectors with L^dag R = I.
 * mu and m_w record the operator the vectors belong to; ovl_sign_apply
 * rejects a solve whose mu/m_w differ. */
int ovl_set_deflation(ovl_lattice lat, double mu, double m_w, int scheme, int m,
                      const double* S_or_R, const double* T, const double* L,
                      ovl_deflation* out);

/* Compute the m critical eigenpairs (smallest |Re lambda|, Sec. 5) on the GPU
 * by restarted Arnoldi (Krylov-Schur) on the same stencil and Gram-Schmidt
 * kernels, and build the deflation data for the scheme. tol: relative
 * residual |A r - lambda r| / (|A|_est |r|) required for every pair;
 * max_restarts bounds the work (OVL_ENOCONV past it). */
int ovl_deflation_setup(ovl_lattice lat, double mu, double m_w, int scheme, int m,
                        double tol, int max_restarts, ovl_deflation* out);
/* ovl_deflation_setup with the caller's choice of polynomial acceleration
 * (not in the paper, which used ARPACK). After one unfiltered expansion on
 * A^2 the solver restarts on C = T_d(l(A^2)), the Chebyshev polynomial of odd
 * degree d in the affine map l that sends the bulk of the spectrum of A^2 (its
 * Ritz values above the 2 nev-th from the left) to [-1, 1]: the wanted
 * eigenvalues become the largest of C, by a factor that grows like
 * exp(d acosh l). C has the eigenvectors of A^2; one application costs d
 * applications of A^2 (2d stencils), which ovl_deflation_stats counts.
 * poly_degree < 0: d chosen from the Ritz values (|T_d| about 1e4 at the
 * leftmost one; this is what ovl_deflation_setup does); 0: plain restarted
 * Arnoldi on A^2 throughout; > 0: that degree (rounded up to odd, at most 201).
 * Convergence on C: every wanted Ritz value theta_i of C with
 * |A^2-coupling b_i| <= tol |theta_i|. */
int ovl_deflation_setup_ex(ovl_lattice lat, double mu, double m_w, int scheme, int m,
                           double tol, int max_restarts, int poly_degree, ovl_deflation* out);

/* Copy the deflation data back (canonical layouts as in ovl_set_deflation;
 * L ignored for Schur). Host or device pointers. */
int ovl_get_deflation(ovl_deflation d, int* scheme, int* m, double* S_or_R, double* T, double* L);
/* Work done by ovl_deflation_setup for this object: restarts of the
 * restarted Arnoldi runs and applications of A^2 (0 for imported data). */
int ovl_deflation_stats(ovl_deflation d, int* restarts, int* matvecs);
int ovl_destroy_deflation(ovl_deflation d);

/* Keep deflation data across processes (not in the paper; Sec. 5 amortises the
 * one-off eigenvector computation over many evaluations). ovl_deflation_save
 * writes the vectors (complex128, canonical layout), T or Lambda, mu, m_w, the
 * setup counts, the lattice dims and boundary and a 64-bit fingerprint of the
 * links (taken by ovl_set_links), followed by a checksum. ovl_deflation_load
 * creates a new object (owned by the caller) on lat and returns OVL_EINVAL when
 * the file is missing, damaged or truncated, or was written for other dims,
 * another boundary condition or other links. Host files; the data go through
 * host memory (2 x 16 x N x m bytes for LR). */
int ovl_deflation_save(ovl_deflation d, const char* path);
int ovl_deflation_load(ovl_lattice lat, const char* path, ovl_deflation* out);

/* ---- the sign function (Secs. 2-4) ------------------------------------- */

/* nsolve independent approximations y_i ~ sgn(H_w(mu_i)) b_i run together
 * (one launch per step for the whole batch; uneven k allowed).
 *  params[i]: mu, m_w, k, precision of solve i.
 *  defl[i]:   deflation data for solve i or NULL (no deflation, Eq. 11);
 *             Schur -> Eq. 19 (computed as Eq. 16 on the block matrix),
 *             LR    -> Eq. 22.  defl may itself be NULL (no solve deflated).
 *  b, y:      nsolve canonical spinors each (stride 24*V doubles).
 *  info:      nsolve records, or NULL.
 * Returns the first non-zero per-solve status (all solves are attempted). */
int ovl_sign_apply(ovl_lattice lat, int nsolve, const ovl_sign_params* params,
                   const ovl_deflation* defl, const double* b, double* y, ovl_sign_info* info);

/* Device workspace (bytes, as a double) that ovl_sign_apply needs for this
 * batch -- Krylov bases of k_max + 1 columns (k when not adaptive), the small
 * matrices and the Newton work -- without running or allocating anything,
 * so that a caller can size batches to the device memory it has (the
 * predictor's admission, predictor.py). The lattice's workspace grows to the
 * largest batch run on it and is kept until ovl_destroy_lattice. Errors as
 * ovl_sign_apply's argument checks. */
int ovl_sign_workspace_bytes(ovl_lattice lat, int nsolve, const ovl_sign_params* params,
                             const ovl_deflation* defl, double* bytes);

/* ---- the overlap operator (Sec. 1, Eq. 1) -------------------------------
 * adjoint = 0: y_i = D_ov(mu_i) x_i = x_i + gamma_5 sgn(H_w(mu_i)) x_i.
 * adjoint = 1: y_i = D_ov(mu_i)^dag x_i = x_i + sgn(H_w(-mu_i)) gamma_5 x_i
 *              (sgn(H_w(mu))^dag = sgn(H_w(-mu)), from Eq. 2); params keep
 *              mu_i, and defl[i] must belong to H_w(-mu_i) (NULL, or from
 *              ovl_deflation_adjoint).
 * The sign runs as in ovl_sign_apply with the same params (info as there);
 * x, y: nsolve canonical spinors, host or device; gamma_5 = diag(1,1,-1,-1) on
 * the spin index. Allocates 3 x nsolve spinors of device work space per call.
 * Errors as ovl_sign_apply; OVL_EINVAL for adjoint not 0 or 1. */
int ovl_overlap_apply(ovl_lattice lat, int nsolve, const ovl_sign_params* params,
                      const ovl_deflation* defl, const double* x, double* y, int adjoint,
                      ovl_sign_info* info);

/* LR deflation data of H_w(-mu) = H_w(mu)^dag from those of H_w(mu) (Eq. 20:
 * left and right eigenvectors swap, eigenvalues are conjugated), for the
 * adjoint overlap operator with one eigenvector computation (Sec. 5). The new
 * object is owned by the caller (ovl_destroy_deflation). OVL_ENOTSUP for
 * Schur data (the Schur vectors of H_w(mu) are not those of its adjoint). */
int ovl_deflation_adjoint(ovl_deflation d, ovl_deflation* out);

/* ---- learned (k, m) predictor (not in the paper) ---------------------- */

/* A small MLP x (n_in) -> ReLU -> ReLU -> y (n_out), FP32 on the device, with
 * its own forward, backward and Adam kernels. It predicts (log k, log(m+1))
 * from solve features so the Krylov basis can be sized before a solve; the
 * adaptive depth of ovl_sign_apply is the fallback. Parameters are one flat
 * vector [W1 (n_h x n_in, row-major), b1, W2, b2, W3, b3]. Loss: mean of
 * w (y - t)^2 with w = under_weight where y < t. Arrays: host or device.
 * n_in <= 32, n_hidden a multiple of 32 in [32, 128], n_out <= 4. */
typedef struct ovl_mlp_s* ovl_mlp;
int ovl_mlp_create(int n_in, int n_hidden, int n_out, ovl_mlp* out);
int ovl_mlp_destroy(ovl_mlp net);
int ovl_mlp_num_params(ovl_mlp net, int* np);
int ovl_mlp_set_params(ovl_mlp net, const float* theta);  /* also resets Adam state */
int ovl_mlp_get_params(ovl_mlp net, float* theta);
int ovl_mlp_forward(ovl_mlp net, const float* X, int batch, float* Y);       /* X: batch x n_in */
int ovl_mlp_loss_grad(ovl_mlp net, const float* X, const float* T, int batch, float under_weight,
                      float* loss, float* grad);                            /* grad: np floats */
int ovl_mlp_train(ovl_mlp net, const float* X, const float* T, int batch, int steps, float lr,
                  float under_weight, float* final_loss);                   /* full-batch Adam */
const char* ovl_mlp_last_error(ovl_mlp net);

/* Features for the predictor. ovl_link_spread: mean over links of
 * 1 - Re tr U / 3. ovl_ritz_values: the k Ritz values of H_w(mu) from k
 * Arnoldi steps (FP64 mode, no deflation) started at b (canonical spinor,
 * host or device); out (host memory) receives k complex128 values. */
int ovl_link_spread(ovl_lattice lat, double* spread);
int ovl_ritz_values(ovl_lattice lat, double mu, double m_w, int k, const double* b, double* out);

/* Kernel accounting for timing reports. ovl_launch_count: kernels launched
 * through this handle so far. ovl_profile(enable=1) clears and starts
 * per-kernel-class CUDA-event timing of ovl_sign_apply on the lattice's
 * stream; enable=0 stops it. stats (may be NULL) receives 8 records of
 * {launches, total milliseconds, algorithmic bytes} for the classes:
 * 0 stencil, 1 Gram-Schmidt pass A, 2 partial-sum reduction, 3 small step,
 * 4 Gram-Schmidt pass B, 5 Newton sign, 6 FP64 projections, 7 recombination. */
int ovl_launch_count(ovl_lattice lat, long long* n);
int ovl_profile(ovl_lattice lat, int enable, double* stats);

/* CUDA graphs for the Arnoldi loop of ovl_sign_apply (not in the paper).
 * enable = 1: a fixed-depth batch (no adaptive depth, no ovl_profile timing)
 * that repeats the shape of the previous call on this handle (same solves,
 * depths, deflation data, mu values and workspace) is captured into a CUDA
 * graph on its second call and replayed on every later one: one graph
 * launch instead of five kernel launches per Arnoldi step. Results are
 * those of the eager launches. A workspace that has to grow drops the graph.
 * enable = 0: off (the default; drops the graph); -1: only query.
 * replays (may be NULL): graph replays on this handle so far. */
int ovl_set_graphs(ovl_lattice lat, int enable, long long* replays);

/* How the Gram-Schmidt update pass (pass B of the Arnoldi step, Eq. 7; the
 * reorthogonalised column and the next candidate) reads the Krylov basis in
 * the 48-bit and 40-bit forms (not in the paper; a load strategy only).
 * bulk = 1: each warp streams its basis columns through a ring of
 * shared-memory stages filled by asynchronous bulk copies ahead of use;
 * bulk = 0 (the default): plain register loads, the faster of the two on
 * GB300 (the per-column bookkeeping of the ring costs more issue slots than
 * the latency it hides). Both give the same results bit for bit.
 * The bulk path needs 16-byte aligned columns and N % 4 == 0 (always true for
 * the library's own workspace); otherwise the register path runs. A stage
 * wait that times out ends the solve with status OVL_ETIMEOUT. Returns
 * OVL_EINVAL for bulk outside {0, 1}. */
int ovl_set_pass_b(ovl_lattice lat, int bulk);

/* Autotuner of the stencil's launch shape (not in the paper). For the FP32
 * stencil with 12-real and with 18-real links and the FP64 stencil, times
 * every candidate shape on this lattice with nrhs right-hand sides (CUDA
 * events, 5 launches after 2 warm-up launches): 128 consecutive sites per CTA
 * (and for FP64 also 32), CTAs covering a tx x ty x tz tile of sites at one t
 * (x fastest; tx*ty*tz = 128, or 32 for FP64; only tiles that divide the
 * lattice), and for FP32 a kernel that stages each hop's neighbour spinor and
 * link in shared memory by asynchronous copies. The fastest shape per (spinor
 * format, link type) is kept in the handle and used by every later stencil
 * launch on it (the FP64 shape also for OVL_LINKS_F64DF); results do not
 * depend on the shape. Allocates 2 x nrhs complex128 spinors of work space for
 * the call. For FP32 also the consecutive-site kernel with its registers
 * capped for 6 and for 4 resident CTAs per SM instead of 8 (fewer spills,
 * fewer warps). report (host, may be NULL): up to max_report records of 8
 * doubles {fmt, links, tpb, tx, ty, tz, variant, microseconds per launch},
 * variant = async (0/1) + 10 x the register cap's CTAs (0: the default 8);
 * *n_report (may be NULL) gets their number. */
int ovl_autotune(ovl_lattice lat, int nrhs, double* report, int max_report, int* n_report);
/* The shape in use for (fmt OVL_VEC_*, links OVL_LINKS_*): {tpb, tx, ty, tz,
 * variant} as in the report; all zero: the built-in rule (consecutive sites, 128 threads; FP64: 32
 * threads on launches of fewer than 1024 sites per SM). */
int ovl_autotune_shape(ovl_lattice lat, int fmt, int links, int shape[5]);
/* Set the shape for (fmt, links) directly (as ovl_autotune_shape reports it);
 * OVL_EINVAL for a tile that does not divide the lattice, a thread count other
 * than 128 (or 32 for FP64), or the staged kernel for FP64 spinors. */
int ovl_autotune_set_shape(ovl_lattice lat, int fmt, int links, const int shape[5]);

/* Failure-detection self test: one CTA waits at a two-member device barrier
 * that nobody else joins, with the same bounded wait the Newton kernel uses
 * (max_polls polls of about 100 ns, at most 2^24). *status receives
 * OVL_ETIMEOUT when the wait gave up as designed; the context stays usable. */
int ovl_wait_selftest(ovl_lattice lat, long long max_polls, int* status);

/* Message for the last failed call on this handle (NULL handle: the last
 * failure of a call that had no handle yet, e.g. ovl_create_lattice). */
const char* ovl_last_error(ovl_lattice lat);

/* Version string of the build ("ovl <semver> sm_103a"). */
const char* ovl_version(void);

#ifdef __cplusplus
}
#endif
#endif /* OVL_H */
