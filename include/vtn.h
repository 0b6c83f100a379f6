/*
 * vtn.h -- C ABI of the GB300 (sm_103a) implementation of the variational tensor-network
 * simulation of Gaussian Boson Sampling (Vinther & Kastoryano, arXiv 2410.18740).
 *
 * The method: the GBS output state |psi> = U V|0> is the unique zero-energy ground state
 * of the parent Hamiltonian H = sum_n A_n^dag A_n (Eq. CentralEquation), which for
 * single-mode squeezers r_k followed by an interferometer U is the quadratic form
 * H = R^T (V^{-1}/4) R - N/2 in the quadratures R = (X_1..X_N, P_1..P_N) with V the
 * covariance matrix (Eq. GBSHamiltonian).  H is written in a truncated Fock basis
 * (Eq. ProjectionOperator: the projected P H P) or in the Gaussian optimal local basis
 * (Eqs. WilliamsonDecomposition, OLB), as a matrix product operator, and its ground
 * state is found as a matrix product state (Eq. MPSAnsatz) by two-site DMRG.  The
 * variational energy <H> >= 0 measures the simulation error (Eq. MagOfSimError).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - hbar = 1, vacuum quadrature variance 1/2, a = (X + iP)/sqrt(2); output modes
 *    a_out = U a_in; squeezer k squeezes X: Var X_k = exp(-2 r_k)/2.
 *  - Complex numbers are stored as interleaved (re, im) pairs of IEEE doubles.
 *    "complex[n]" below means 2n doubles.
 *  - Tensors are row-major.  MPS site tensor A[a][s][b] (left bond, physical, right
 *    bond).  Left environment L[w][bra][ket], right environment R[w][ket][bra].  MPO
 *    core W[a][b][s'][s] = <s'|op_ab|s>.
 *  - Ownership: the caller owns every array it passes; the library copies what it
 *    keeps.  The library owns vtn_ctx / vtn_mpo / vtn_mps handles; they are released
 *    only by the matching *_free / vtn_destroy call.  Output arrays are allocated by
 *    the caller.  Pointers documented as "device" must be device memory of the
 *    context's GPU; all others are host memory.
 *  - Streams: all device work of a context runs on the stream given to vtn_create
 *    (NULL = the legacy default stream).  Calls that write host outputs synchronise
 *    that stream before returning; calls whose outputs are device arrays are
 *    asynchronous with respect to the host and ordered on the stream.
 *  - Errors: every call returns a vtn_status and never aborts or exits.  On failure
 *    the out-parameters are left untouched (vtn_sweep keeps the last valid MPS) and
 *    vtn_last_error(ctx) holds a one-line message.
 *  - Threads: one context per host thread.
 */
#ifndef VTN_H
#define VTN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vtn_ctx_s* vtn_ctx;
typedef struct vtn_mpo_s* vtn_mpo;
typedef struct vtn_mps_s* vtn_mps;
typedef struct vtn_mlp_s* vtn_mlp;

typedef enum {
    VTN_OK = 0,
    VTN_EINVAL = 1,        /* invalid argument (sizes, non-unitary U, d > D, ...)        */
    VTN_ENOMEM = 2,        /* device or host allocation failed                           */
    VTN_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed                */
    VTN_ENOCONV = 4,       /* Lanczos missed its tolerance after all restarts; the best
                              Ritz vector was still used                                 */
    VTN_ETIMEOUT = 5,      /* a bounded device-side wait gave up                         */
    VTN_EUNSUPPORTED = 6   /* a valid request outside what this build implements         */
} vtn_status;

typedef enum {
    VTN_FP64 = 0,          /* every contraction in IEEE double (SIMT FP64 FMA)           */
    VTN_TF32X3 = 1,        /* reserved: three-term TF32 split products (VTN_EUNSUPPORTED) */
    VTN_BF16X3 = 2         /* H_eff psi and the environment updates on the tensor cores:
                              each FP64 operand split into bf16 hi + lo, products
                              hi*hi + hi*lo + lo*hi accumulated in FP32 (relative error
                              ~1e-5 per product); the MPO mixing between the GEMMs in
                              FP32; environments stored in FP64.  Lanczos, the truncation
                              eigendecomposition and energies stay FP64. */
} vtn_precision;

/* Optional device-memory provider.  alloc returns device memory of at least `bytes`
 * bytes aligned to 256 B on the context's device, or NULL on failure; free releases
 * it.  With no provider the library calls cudaMalloc / cudaFree. */
typedef struct {
    void* (*alloc)(size_t bytes, void* user);
    void (*free)(void* ptr, void* user);
    void* user;
} vtn_allocator;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` whose work runs on `cuda_stream`
 * (a cudaStream_t, NULL = legacy default stream).  `allocator` may be NULL. */
vtn_status vtn_create(vtn_ctx* out, int device, void* cuda_stream, const vtn_allocator* allocator);
vtn_status vtn_destroy(vtn_ctx ctx);
/* Last error message of the context ("" if none).  Valid until the next call on ctx.
 * vtn_last_error(NULL) returns the message of the calling thread's last failed call made
 * without a context (vtn_create, the host-only MPO builders and queries). */
const char* vtn_last_error(vtn_ctx ctx);
/* Number of kernels this context has launched since creation (all entry points). */
vtn_status vtn_launch_count(vtn_ctx ctx, long long* out);

/* ---------------------------------------------------------------- problem -> MPO */

#define VTN_FLAG_LBO 1u    /* force the Gaussian optimal local basis even when d == D */

/* Build the MPO of the GBS parent Hamiltonian (Eq. GBSHamiltonian) and upload it.
 *   M  >= 1 modes; r: double[M] squeezing parameters; U: complex[M*M] row-major
 *      interferometer with a_out = U a_in (validated: max |U^dag U - I| <= 1e-10).
 *   D  >= 2 physical Fock cutoff (Eq. ProjectionOperator).
 *   d  local dimension of the solver, 1 <= d <= D, d <= 16.  d == D (and no
 *      VTN_FLAG_LBO): Fock basis.  Otherwise each mode is rotated to its optimal local
 *      basis S_i^dag|m> from the Williamson decomposition of its reduced covariance
 *      (Eqs. WilliamsonDecomposition, OLB) and the D x d isometry
 *      V_nm = <n|S_i^dag|m> (Eq. InverseBasisTransformation) is kept for read-out.
 * Same-mode operator products are exactly projected (P H P; SM Sec. 5).
 * The MPO is the centre-collapsed state machine of SM Sec. 8 (Gaussian part):
 * bond dimension w_s = 2 min(s, M - s) + 2 inside, 1 at the ends. */
vtn_status vtn_build_mpo(vtn_ctx ctx, int M, const double* r, const double* U,
                         int D, int d, unsigned flags, vtn_mpo* out);

/* Build the MPO of the non-Gaussian workload of Sec. "Beyond GBS: fully connected CZ-gate":
 * |psi> = exp(-i kappa prod_k X_k)|psi_G> (Eq. GlobalCZgate) for the Gaussian state of
 * (r, U), whose parent Hamiltonian (Eq. nonGBSHamiltonian, zero means) is
 * H = R'^T (V^-1/4) R' - N/2 with R' = (X, P + xi), xi_i = kappa prod_{n != i} X_n.
 * Fock basis only (the local dimension is D; no optimal local basis); M >= 2; r, U, D
 * validated as for vtn_build_mpo; kappa finite (kappa = 0 gives the GBS MPO).  Same-mode
 * products are exactly projected.  The MPO is the Gaussian one with, at every inner cut s,
 * 4 + 4s channels appended for the kappa and kappa^2 terms (full-chain products of X or X^2
 * with at most two special modes).  Everything else (vtn_sweep, vtn_energy, marginals,
 * sampling, vtn_energy_variance) accepts the result like any MPO. */
vtn_status vtn_build_mpo_cz(vtn_ctx ctx, int M, const double* r, const double* U, int D, double kappa,
                            vtn_mpo* out);
/* Closed-form bond spectrum of the Gaussian state the MPO describes: the k largest
 * eigenvalues (descending, zero-padded) of the reduced state of modes 0..cut-1, i.e. the
 * squared Schmidt values of the cut, prod_j (1 - q_j) q_j^{n_j} with q_j = nbar_j/(nbar_j + 1),
 * nbar_j = nu_j - 1/2 and nu_j the symplectic eigenvalues of the block's covariance (the
 * multi-mode form of Eq. diagReducedGaussianDM).  Infinite Fock cutoff: the ground state of
 * P H P approaches it as D grows (local bases leave it unchanged).  out: host double[k].
 * VTN_EUNSUPPORTED for MPOs without a Gaussian state (given as cores, or kappa != 0).  Host only. */
vtn_status vtn_gaussian_bond_spectrum(vtn_mpo mpo, int cut, int k, double* out);
/* Per cut s = 0..M, the smallest bond dimension whose discarded weight in that closed-form
 * spectrum is <= eps, capped at min(chi_max, d^s, d^(M-s)) (at least 1).  dims: host int[M+1]. */
vtn_status vtn_gaussian_bond_dims(vtn_mpo mpo, double eps, int chi_max, int* dims);
vtn_status vtn_mpo_free(vtn_mpo mpo);
/* Shape queries: M, d, D and the bond dimensions w[0..M] (w may be NULL). */
vtn_status vtn_mpo_info(vtn_mpo mpo, int* M, int* d, int* D, int* w);
/* Coefficient matrix of the quadratic form actually used, G = V^{-1}/4 (xxpp order),
 * or G' = S^T G S in the optimal local basis: double[2M*2M]. */
vtn_status vtn_mpo_coefficients(vtn_mpo mpo, double* G);
/* Covariance matrix V (xxpp order): double[2M*2M]. */
vtn_status vtn_mpo_covariance(vtn_mpo mpo, double* V);
/* Isometry of mode `site` (complex[D*d], row n, column m); identity block in the Fock
 * basis.  Its global phase is a convention: probabilities do not depend on it. */
vtn_status vtn_mpo_isometry(vtn_mpo mpo, int site, double* V);
/* Sparse entries of core `site`: *nnz on input is the capacity of rows/cols/ops, on
 * output the count.  ops: complex[nnz*d*d], ops[k][s'][s].  Passing rows == NULL
 * returns only the count. */
vtn_status vtn_mpo_core(vtn_mpo mpo, int site, int* nnz, int* rows, int* cols, double* ops);
/* Term form of the two-site H_eff of bond (bond, bond+1) used by the split-precision sweeps
 * (host query, no device needed).  Each core's d x d entries are expanded in an operator basis
 * (Bi: ri operators of core `bond`, Bj: rj of core `bond + 1`, each d x d with [0] = I), and
 *   H_eff = sum_t (sum_a U[t][a] L[a]) (x) (Bi[o_t] (x) Bj[p_t]) (x) (sum_c V[t][c] R[c])
 * exactly (up to rounding) for the environments L[a] (a < w[bond]) and R[c] (c < w[bond+2]) of
 * Sec. "Matrix Product States"; the first n_id terms have o_t = p_t = 0.  Call with ops == NULL to
 * get *usable, *n_terms, *n_id, *ri, *rj; then ops int[2 n_terms] (o_t, p_t), U complex[n_terms
 * w[bond]], V complex[n_terms w[bond+2]], Bi complex[ri d d], Bj complex[rj d d] (row = output
 * level).  *usable = 1: the sweeps use the term form at this bond; 2: the bond has one, but with
 * more than 1.15 max(w_l, w_r) + 4 terms the channel-mixing form is cheaper and is used; 0 (and
 * n_terms = 0): no compact term form (an operator basis of 16 or more elements, or d > 8).  A
 * sweep factorises and uploads a bond's term form on the bond's first split-precision use (a few
 * milliseconds of host work a bond); vtn_sweep_batch does so for every bond before it starts. */
vtn_status vtn_mpo_bond_terms(vtn_mpo mpo, int bond, int* usable, int* n_terms, int* n_id, int* ri, int* rj,
                              int* ops, double* U, double* V, double* Bi, double* Bj);
/* Deterministic bound ||P H P|| <= lambda_max(G) M (2d - 1), used to scale tolerances. */
vtn_status vtn_mpo_norm_bound(vtn_mpo mpo, double* out);

/* ---------------------------------------------------------------- MPS */

/* Seeded random right-canonical MPS with bond dimensions min(chi, d^s, d^(M-s)):
 * entry j of site s is the complex normal (g1 + i g2)/sqrt(2) drawn by Box-Muller from
 * Philox4x32-10 (key = seed, counter = (j, site, 1)); the rows of every site matrix
 * (left bond) x (physical, right bond) are then orthonormalised in order. */
vtn_status vtn_mps_random(vtn_ctx ctx, vtn_mpo mpo, int chi, uint64_t seed, vtn_mps* out);
/* MPS from host tensors: dims[0..M] bond dimensions (dims[0] = dims[M] = 1), sites[s]
 * complex[dims[s]*d*dims[s+1]].  No canonical form is assumed. */
vtn_status vtn_mps_from_host(vtn_ctx ctx, vtn_mpo mpo, const int* dims, const double* const* sites,
                             vtn_mps* out);
/* The same draws as vtn_mps_random in mixed-canonical form with the orthogonality centre at
 * site `center` (0 <= center < M): sites s < center get the columns of their (left bond,
 * physical) x (right bond) matrix orthonormalised in order (left-canonical), sites s >= center
 * the rows (right-canonical), and the centre site is then divided by sqrt(dims[center]) so
 * that <psi|psi> = 1.  center = 0 is vtn_mps_random. */
vtn_status vtn_mps_random_center(vtn_ctx ctx, vtn_mpo mpo, int chi, uint64_t seed, int center, vtn_mps* out);
/* The orthogonality centre the library records for an MPS: the site whose left neighbours are
 * all left-canonical and right neighbours all right-canonical, or -1 when unknown (an MPS
 * from host tensors).  Sweeps and vtn_mps_move_center keep it up to date. */
vtn_status vtn_mps_get_center(vtn_mps mps, int* center);
/* Record the centre of an MPS whose tensors the caller built in that gauge (not checked), or
 * forget it (center = -1).  -1 <= center < M. */
vtn_status vtn_mps_set_center(vtn_mps mps, int center);
/* Move the orthogonality centre to `center` (0 <= center < M) by exact splits of neighbouring
 * sites: theta = A_i A_i+1 is split by the FP64 reduced-density-matrix eigendecomposition of
 * vtn_truncate keeping k = the current bond dimension (no state is dropped, so psi is
 * unchanged up to rounding and a gauge transformation).  An MPS with an unknown centre is
 * first brought to centre 0 by splits from the right end. */
vtn_status vtn_mps_move_center(vtn_ctx ctx, vtn_mps mps, int center);
vtn_status vtn_mps_free(vtn_mps mps);
vtn_status vtn_mps_info(vtn_mps mps, int* M, int* d, int* dims);
/* Copy site s to host: complex[dims[s]*d*dims[s+1]]. */
vtn_status vtn_mps_get_site(vtn_ctx ctx, vtn_mps mps, int site, double* out);
/* Flat binary checkpoint: magic, M, d, dims, tensors. */
vtn_status vtn_mps_save(vtn_ctx ctx, vtn_mps mps, const char* path);
vtn_status vtn_mps_load(vtn_ctx ctx, vtn_mpo mpo, const char* path, vtn_mps* out);

/* ---------------------------------------------------------------- solver */

typedef struct {
    int chi_max;               /* maximum bond dimension                                 */
    const int* chi_schedule;   /* per-sweep chi (growth from O(1), Discussion); NULL = chi_max */
    int n_schedule;
    int n_sweeps;              /* maximum number of sweeps (<= 64)                       */
    vtn_precision prec;        /* contraction precision of H_eff psi and environments    */
    double lanczos_tol;        /* absolute residual ||H x - theta x|| to stop Lanczos     */
    int krylov_max;            /* Krylov dimension before an explicit restart (<= 64)    */
    int lanczos_max_restarts;
    double e_tol;              /* stop when |E_k - E_{k-1}| <= e_tol (0 = off)            */
    double e_target;           /* stop when E_k <= e_target (used when use_e_target != 0) */
    int use_e_target;
    uint64_t seed;             /* seed of the random initial MPS when *state == NULL      */
    int trunc_mode;            /* 0: exact eigendecomposition (the paper's truncation);
                                  1: warm-started subspace iteration (vtn_truncate_warm)   */
    int trunc_q;               /* subspace iterations of trunc_mode 1 (0..64)            */
    int window_lo, window_hi;  /* window_hi > window_lo: a windowed sweep over the bonds
                                  window_lo .. window_hi - 1 only (0 <= lo < hi <= M - 1)   */
    int energy_mode;           /* energy reported after each sweep: 0 = full FP64 contraction
                                  <psi|H|psi>/<psi|psi>; 1 = Rayleigh quotient of the final
                                  centre tensor (windowed sweeps always use 1)            */
    int heff_form;             /* split-precision H_eff psi: 0 = the term form where the bond
                                  has one and it is the cheaper form (cores folded into the
                                  environments once per bond, see vtn_mpo_bond_terms), else
                                  the channel-mixing form; 1 = the channel-mixing form always;
                                  2 = the term form wherever the bond has one               */
    int env_fp64;              /* with prec = VTN_BF16X3: 1 = environment updates in FP64 (their
                                  split-precision errors add up along the chain: about 5e-4
                                  relative after 49 updates at chi = 256, see
                                  vtn_set_tc_accumulation); 0 = split precision as H_eff psi */
} vtn_sweep_opts;

typedef struct {
    int sweeps_done;
    double energy[64];         /* FP64 <H> of the normalised MPS after each sweep         */
    double max_discarded[64];  /* largest discarded weight of the sweep (Eq. SurrogateEpsChi) */
    double seconds[64];        /* wall time of each sweep                                */
    long long matvecs;         /* H_eff psi products                                      */
    long long lanczos_not_converged;
    double heff_flops;         /* algorithmic real flops of all H_eff psi products        */
    double heff_seconds;       /* device time of the H_eff psi GEMM launches (timing on)  */
    double gemm_flops;         /* algorithmic real flops of every complex GEMM launch     */
    double gemm_seconds;       /* their device time (timing on)                           */
    double eig_seconds;        /* device time of the truncation eigensolver (timing on)   */
    long long host_syncs;      /* times the call waited for the GPU (stream synchronisations):
                                  with lanczos_max_restarts = 0 and the exact truncation, once
                                  per sweep plus set-up and workspace growth; otherwise also
                                  once per Lanczos step and per truncation                  */
} vtn_sweep_report;

/* Fill opts with the defaults: chi_max 16, 8 sweeps, FP64, lanczos_tol 1e-10,
 * krylov_max 32, 4 restarts, e_tol 0, seed 0, trunc_mode 0 (exact), trunc_q 1, no window,
 * energy_mode 0, heff_form 0, env_fp64 0. */
vtn_status vtn_sweep_opts_default(vtn_sweep_opts* opts);

/* Two-site DMRG sweeps.  *state == NULL: start from vtn_mps_random(opts->chi_schedule[0]
 * or chi_max, opts->seed).  A sweep optimises bonds (0,1) .. (M-2,M-1) left to right,
 * then (M-2,M-1) .. (0,1) right to left; it ends right-canonical with the centre at
 * site 0.  Each bond: Lanczos on H_eff (full re-orthogonalisation, restarts), FP64
 * eigendecomposition of the reduced density matrix, keep min(chi, chi_l d, d chi_r)
 * largest eigenpairs, environment update.  A state whose recorded orthogonality centre is a
 * site other than 0 is first brought back to centre 0 (vtn_mps_move_center).
 * Windowed sweep (opts->window_hi > opts->window_lo): each sweep optimises bonds
 * (lo,lo+1) .. (hi-1,hi) left to right, then back to (lo,lo+1), and ends with the centre at
 * site lo; the state is first moved to centre lo if its recorded centre is elsewhere
 * (sites < lo must be left-canonical, sites > lo right-canonical for the environments).
 * Only the environments the window needs are built.  Its sweep energy is always the
 * Rayleigh quotient of the final centre (energy_mode 1): <theta|H_eff theta>/<theta|theta>
 * for theta = A_lo A_lo+1 and the H_eff of bond (lo, lo+1) in the sweep's contraction
 * precision, FP64 sums; for a canonical state this is <psi|H|psi>/<psi|psi> (Eq.
 * MagOfSimError) without a contraction over the whole chain.  With opts->trunc_mode = 1 the truncation is
 * vtn_truncate_warm with q = opts->trunc_q, p = 8, seed = opts->seed, bond = i and the
 * current centre tensor (site i sweeping right, site i+1 sweeping left) as start vectors.
 * Returns VTN_ENOCONV (after finishing) if some Lanczos solve missed its tolerance.  report
 * may be NULL. */
vtn_status vtn_sweep(vtn_ctx ctx, vtn_mpo mpo, vtn_mps* state, const vtn_sweep_opts* opts,
                     vtn_sweep_report* report);

/* Independent two-site sweeps of n instances at once (many GBS instances of uneven size):
 * instance j runs vtn_sweep(mpos[j], &states[j], &opts[j], &reports[j]) (reports may be NULL),
 * status[j] gets its result.  The instances are spread over n_streams worker contexts (1..64),
 * each with its own CUDA stream and workspace and a host thread that takes the next instance
 * when its current one is done, so that the kernels of different instances overlap on the GPU
 * (the small-bond instances leave most SMs idle alone).  States that are NULL are created first
 * (vtn_mps_random with opts[j]'s first bond dimension and seed) on ctx; the MPOs and states stay
 * owned by ctx.  Results equal the one-by-one vtn_sweep calls.  Returns the first error of an
 * instance, else VTN_ENOCONV if some instance returned it, else VTN_OK; the workers are released
 * before returning. */
vtn_status vtn_sweep_batch(vtn_ctx ctx, int n, const vtn_mpo* mpos, vtn_mps* states, const vtn_sweep_opts* opts,
                           vtn_sweep_report* reports, vtn_status* status, int n_streams);

/* Single-site DMRG with subspace expansion: the solver of the paper's results section
 * (single-site DMRG), with the bond dimension grown during the sweeps as its discussion
 * describes, by the strictly single-site expansion it cites (Hubig et al., Phys. Rev. B 91,
 * 155115 (2015)).  FP64 only (opts->prec other than VTN_FP64: VTN_EUNSUPPORTED); the other
 * opts fields as for vtn_sweep.  A sweep optimises sites 0 .. M-2 left to right, then
 * M-1 .. 1 right to left, and ends with the centre on site 0.  At site i moving right:
 *   1. Lanczos on y[l,t,r'] = sum L[a,l,l'] W_i[a,b,t,s] A[l',s,r] R[b,r,r'] (A = site i);
 *   2. expansion Mx = [A | alpha_t P], P[(l t), (b r)] = sum L[a,l,l'] W_i[a,b,t,s] A[l',s,r],
 *      a (chi_l d) x chi_r (1 + w_r) matrix (the next site gains zero rows: state unchanged);
 *   3. FP64 eigendecomposition of Mx Mx^dag keeping k = min(chi, chi_l d, chi_r (1 + w_r),
 *      d chi_{i+2}) eigenpairs, then only those with eigenvalue > cutoff * the largest;
 *   4. site i <- U_k (left-canonical), site i+1 <- (U_k^dag A) site i+1, L_{i+1} updated.
 * Moving left mirrors it (Mx = [A; alpha_t P], P[(a l), (t r')] = sum W_i[a,b,t,s] A[l,s,r]
 * R[b,r,r']).  alpha_t = alpha * alpha_decay^t in sweep t (alpha >= 0, alpha_decay >= 0);
 * cutoff in [0, 1).  Without the expansion (alpha = 0) the bonds never grow.  report as for
 * vtn_sweep (heff_flops: 8 d chi_l chi_r (w_l chi_l + w_r chi_r) per product); returns
 * VTN_ENOCONV (after finishing) if some Lanczos solve missed its tolerance. */
vtn_status vtn_sweep_single_site(vtn_ctx ctx, vtn_mpo mpo, vtn_mps* state, const vtn_sweep_opts* opts,
                                 double alpha, double alpha_decay, double cutoff, vtn_sweep_report* report);

/* <psi|H|psi> / <psi|psi> in FP64 by a full environment contraction (Eq. MagOfSimError). */
vtn_status vtn_energy(vtn_ctx ctx, vtn_mpo mpo, vtn_mps mps, double* E);

/* Energy variance of the variational state (Sec. "Assessing the error from finite bond
 * dimension": sigma_H = sqrt(<(PHP)^2> - <PHP>^2), the compression-error estimate; sigma_H
 * near 0 means the bond dimension is adequate).  Outputs (each may be NULL):
 * E = <psi|H|psi>/<psi|psi>, H2 = <psi|H H|psi>/<psi|psi>, sigma = sqrt(max(0, H2 - E^2)),
 * all FP64, H being the MPO's operator (the projected P H P).  Cost: two-layer environments of
 * w_s^2 chi_s^2 complex per cut, 16 w^2 chi^3 d flops per site; returns VTN_EINVAL when the
 * device buffers would exceed 24 GiB. */
vtn_status vtn_energy_variance(vtn_ctx ctx, vtn_mpo mpo, vtn_mps mps, double* E, double* H2, double* sigma);

/* Joint photon-number distribution of the k distinct modes `modes` in the Fock basis
 * (after the inverse basis transformation, Eq. InverseBasisTransformation):
 * out: double[D^k], index sum_j n_j D^(k-1-j) in the order of `modes`.  Normalised by
 * <psi|psi> of the solver basis, so with a local basis the D^k values sum to <= 1.
 * VTN_EINVAL if k < 1, a mode repeats or is out of range, or D^k > 2^26. */
vtn_status vtn_marginals(vtn_ctx ctx, vtn_mpo mpo, vtn_mps mps, const int* modes, int k, double* out);
/* Every single-mode marginal: out double[M*D], row i = P_i(n), n < D. */
vtn_status vtn_marginals_all(vtn_ctx ctx, vtn_mpo mpo, vtn_mps mps, double* out);

/* n_samples photon-number patterns by sequential conditional sampling in the Fock
 * basis: p(n_i | n_<i) from the chain rule on the MPS; mode i of sample t takes the
 * smallest n with CDF(n) > u * CDF(D-1), u the 53-bit uniform of Philox4x32-10
 * (key = seed, counter = (t, i, 2)).  out: int32[n_samples*M]. */
vtn_status vtn_sample(vtn_ctx ctx, vtn_mpo mpo, vtn_mps mps, uint64_t seed, int n_samples, int32_t* out);

/* Single-mode reduced density matrix of the variational state, rho_i = Tr_{others} |psi><psi| /
 * <psi|psi> in the solver basis (the partial trace of the read-out, Eq. InverseBasisTransformation
 * applies to it as V rho_i V^dag): out complex[d*d], out[s][t] = <s|rho_i|t>. */
vtn_status vtn_reduced_density(vtn_ctx ctx, vtn_mpo mpo, vtn_mps mps, int site, double* out);

/* Product MPS (every bond dimension 1) with site s = amps[s] / |amps[s]| (amps: host complex[M*d],
 * each site vector non-zero); its recorded centre is 0. */
vtn_status vtn_mps_product(vtn_ctx ctx, vtn_mpo mpo, const double* amps, vtn_mps* out);

/* ---------------------------------------------------------------- kernel-level calls
 * These expose single steps of the solver on caller-provided device buffers.  They
 * are what the solver runs internally and serve parity tests and kernel timing. */

/* Host description of one sparse MPO core: nnz entries (rows[k], cols[k]) with
 * operators ops[k] = complex[d*d] (ops[k][s'][s]), w_left x w_right channels. */
typedef struct {
    int w_left, w_right, d, nnz;
    const int* rows;
    const int* cols;
    const double* ops;
} vtn_core;

/* An MPO given as its cores: cores[s] for s = 0..M-1 (vtn_core), with
 * cores[0].w_left = cores[M-1].w_right = 1, cores[s].w_right = cores[s+1].w_left and one d
 * for all.  For Hamiltonians other than the built-in workloads (and for checks that need a
 * given MPO representation, which the single-site expansion depends on).  The basis is the
 * local basis of the cores (no local-basis isometry: D = d); vtn_mpo_coefficients and
 * vtn_mpo_covariance return VTN_EUNSUPPORTED and vtn_mpo_norm_bound returns 0 (unknown).
 * The library copies the cores.  ctx may be NULL (host-only, uploaded on first use). */
vtn_status vtn_mpo_from_cores(vtn_ctx ctx, int M, const vtn_core* cores, vtn_mpo* out);

/* Two-site effective-Hamiltonian product (the hot path):
 *   y[i,t,u,l] = sum L[a,i,j] Wi[a,b,t,s] Wj[b,c,u,v] theta[j,s,v,k] R[c,k,l]
 * L: device complex[Wi.w_left*chi_l*chi_l]; R: device complex[Wj.w_right*chi_r*chi_r];
 * theta, y: device complex[chi_l*d*d*chi_r].  y must not alias theta. */
vtn_status vtn_heff_apply(vtn_ctx ctx, const vtn_core* Wi, const vtn_core* Wj, int chi_l, int chi_r,
                          const double* L, const double* R, const double* theta, double* y,
                          vtn_precision prec);

/* Environment update across one site with tensor A (device complex[chi_l*d*chi_r]):
 *  side 0 (left):  out[b,l,k] = sum conj(A[i,t,l]) env[a,i,j] W[a,b,t,s] A[j,s,k]
 *                  env: complex[W.w_left*chi_l*chi_l] -> out: complex[W.w_right*chi_r*chi_r]
 *  side 1 (right): out[b,j,i] = sum W[b,c,t,s] A[j,s,g] conj(A[i,t,p]) env[c,g,p]
 *                  env: complex[W.w_right*chi_r*chi_r] -> out: complex[W.w_left*chi_l*chi_l]
 * prec VTN_FP64: FP64 contractions; VTN_BF16X3: both dense contractions as split-precision
 * bf16 products on the tensor cores with FP32 accumulation, FP32 mixing, FP64 output (the
 * mode vtn_sweep uses for its environments when opts->prec is VTN_BF16X3). */
vtn_status vtn_env_update(vtn_ctx ctx, const vtn_core* W, int side, int chi_l, int chi_r,
                          const double* env, const double* A, double* out, vtn_precision prec);

/* Single-site effective-Hamiltonian product (step 1 of vtn_sweep_single_site):
 *   y[l,t,r'] = sum L[a,l,l'] W[a,b,t,s] A[l',s,r] R[b,r,r']
 * L: device complex[W.w_left*chi_l*chi_l]; R: device complex[W.w_right*chi_r*chi_r];
 * A, y: device complex[chi_l*d*chi_r]; y must not alias A.  FP64. */
vtn_status vtn_heff1_apply(vtn_ctx ctx, const vtn_core* W, int chi_l, int chi_r, const double* L,
                           const double* R, const double* A, double* y);

/* Subspace expansion of a centre tensor A (device complex[chi_l*d*chi_r]), step 2 of
 * vtn_sweep_single_site, FP64:
 *  side 0: env = L (complex[W.w_left*chi_l*chi_l]); out = Mx, complex[(chi_l d) x chi_r (1 + W.w_right)],
 *          row (l t), column r < chi_r: A[l,t,r]; column chi_r (1 + b) + r:
 *          alpha sum L[a,l,l'] W[a,b,t,s] A[l',s,r].
 *  side 1: env = R (complex[W.w_right*chi_r*chi_r]); out = Mx, complex[chi_l (1 + W.w_left) x (d chi_r)],
 *          row l < chi_l: A[l,:,:]; row chi_l (1 + a) + l, column (t r'):
 *          alpha sum W[a,b,t,s] A[l,s,r] R[b,r,r'].
 * out must not alias env or A. */
vtn_status vtn_expand(vtn_ctx ctx, const vtn_core* W, int side, int chi_l, int chi_r, const double* env,
                      const double* A, double alpha, double* out);

/* Lowest eigenpair of the two-site H_eff by the solver's Lanczos (full
 * re-orthogonalisation, restarts).  theta: device complex[chi_l*d*d*chi_r], start vector
 * on input, normalised Ritz vector on output.  E: host double.  n_matvec: host, may be
 * NULL.  Returns VTN_ENOCONV if the tolerance was missed. */
vtn_status vtn_heff_ground(vtn_ctx ctx, const vtn_core* Wi, const vtn_core* Wj, int chi_l, int chi_r,
                           const double* L, const double* R, double* theta, double tol,
                           int krylov_max, int max_restarts, double* E, int* n_matvec);

/* Truncation of a two-site tensor theta (device complex[chi_l*d1*d2*chi_r]) viewed as
 * the (chi_l d1) x (d2 chi_r) matrix T, by the FP64 eigendecomposition of the reduced
 * density matrix, keeping k = min(k_max, chi_l d1, d2 chi_r) eigenpairs of largest
 * eigenvalue (squared Schmidt values, Eq. SurrogateEpsChi):
 *  direction 0: rho = T T^dag = U diag(lam) U^dag; left = U_k (chi_l,d1,k, left-canonical),
 *               right = U_k^dag T (k,d2,chi_r).
 *  direction 1: rho = T^dag T = V diag(lam) V^dag; left = T V_k (chi_l,d1,k),
 *               right = V_k^dag (k,d2,chi_r, right-canonical).
 * left/right: device buffers of chi_l*d1*k and k*d2*chi_r complex.  lam: host double[k]
 * (descending), discarded: host double = 1 - sum(kept)/tr(rho).  *k_out = k. */
vtn_status vtn_truncate(vtn_ctx ctx, int chi_l, int d1, int d2, int chi_r, int direction, int k_max,
                        const double* theta, double* left, double* right, double* lam,
                        double* discarded, int* k_out);

/* The same split as vtn_truncate with the kept subspace found by block subspace iteration
 * instead of the full eigendecomposition (not the paper's truncation, which is exact: a
 * cheaper alternative, compared with it by the energies it leads to).  With n = chi_l d1
 * (direction 0, rho = T T^dag) or d2 chi_r (direction 1, rho = T^dag T), k = min(k_max,
 * chi_l d1, d2 chi_r) and m = min(chi_l d1, d2 chi_r, k + p) (no more than the rank of rho):
 *   start vectors: the k0 columns of Q0 (device complex[n*k0], row-major n x k0; in a sweep the
 *   current centre tensor), then rho Omega for the remaining m - k0, Omega (n x (m - k0),
 *   row-major) complex normals (g1 + i g2)/sqrt(2) of Philox4x32-10 with key seed and counter
 *   (j, bond, 3) for entry j; Gram-Schmidt in order (a vector numerically dependent on the ones
 *   before it -- residual below 1e-10 of its norm -- is replaced by an orthonormal completion);
 *   q times: multiply by rho and re-orthonormalise; Rayleigh-Ritz: the k largest eigenpairs (w, Y) of Q^dag rho Q give the
 *   kept vectors Q Y.  rho is applied as T (T^dag X), never formed.  Outputs as vtn_truncate,
 *   with the Ritz values w in lam and discarded = 1 - sum(w)/||T||^2.  0 <= q <= 64,
 *   0 <= p <= 256, m <= 4096, k0 >= 0 (Q0 may be NULL when k0 = 0). */
vtn_status vtn_truncate_warm(vtn_ctx ctx, int chi_l, int d1, int d2, int chi_r, int direction, int k_max,
                             const double* theta, const double* Q0, int k0, int q, int p, uint64_t seed,
                             int bond, double* left, double* right, double* lam, double* discarded, int* k_out);

/* Inverse basis transformation on one site (Eq. InverseBasisTransformation):
 * out[a][n][b] = sum_m V[n][m] A[a][m][b], V device complex[D*d], A device
 * complex[chi_l*d*chi_r], out device complex[chi_l*D*chi_r]. */
vtn_status vtn_lbo_rotate(vtn_ctx ctx, int chi_l, int d, int D, int chi_r, const double* V,
                          const double* A, double* out);

/* H_eff psi for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a facility of the library, not a step of the method.
 *
 * Who it is for: code that must not call cudaMalloc -- for example an application that
 * owns every byte of GPU memory through its own pool under a fixed budget, or a
 * latency-critical loop in which cudaMalloc / cudaFree (which can synchronise the whole
 * device) are not acceptable.  It needs no vtn_ctx (creating one allocates) and allocates
 * nothing: the caller passes inputs and outputs, and every intermediate lives in one
 * file-scope device array of 32 MiB that every GPU which loads the library keeps until the
 * process exits.
 *
 * Same contraction, layouts and argument meaning as vtn_heff_apply (FP64):
 *   y[i,t,u,l] = sum L[a,i,j] Wi[a,b,t,s] Wj[b,c,u,v] theta[j,s,v,k] R[c,k,l]
 * Limits (larger requests return VTN_EINVAL before any work is queued): d <= 16;
 * w_left, w_right <= 512 and nnz <= 4096 for each core; the two cores together need at most
 * 1 MiB of device storage (about nnz * d * d * 16 bytes each); and
 * max(Wi.w_left, Wi.w_right, Wj.w_right) * chi_l * d * d * chi_r <= 1,015,808.
 * Set-up: the first call on a device looks up the array's device address with that device
 * current; make that first call before any stream capture.
 * Sharing: all calls use the same array, which keeps what the previous call left (each call
 * writes every element before reading it, so nothing needs clearing).  Calls whose GPU work
 * overlaps -- on different streams or from different host threads -- race on the array:
 * serialise them.
 * cuda_stream: cudaStream_t the work is queued on (NULL = legacy default stream).  The call
 * returns once the work is queued; the cores' host arrays may be reused immediately.
 * L, R, theta, y: device pointers as for vtn_heff_apply; y must not alias theta.
 * Errors: VTN_EINVAL (limits, null or aliased pointers, inconsistent cores), VTN_ECUDA
 * (symbol lookup, copy or launch failure).  No message is recorded (vtn_last_error does
 * not apply: there is no context). */
vtn_status vtn_heff_apply_static(const vtn_core* Wi, const vtn_core* Wj, int chi_l, int chi_r,
                                 const double* L, const double* R, const double* theta, double* y,
                                 void* cuda_stream);

/* ---------------------------------------------------------------- learned warm start
 * The multilayer perceptron the warm start trains and evaluates (the paper has no learned
 * component; the network maps instance features to solver inputs, and the variational energy
 * they lead to measures its quality).  FP32 on the device: layers n_in -> width (x depth) -> n_out, ReLU after
 * every layer but the last, mean-squared-error loss, Adam (beta1 0.9, beta2 0.999, eps 1e-8;
 * Kingma and Ba 2015).  Parameters are one float array: per layer l, W_l (n_out_l x n_in_l,
 * row-major) then b_l (n_out_l).  x: device float[batch*n_in], t and y: device float[batch*n_out],
 * row-major.  Every call runs on the context's stream and returns after it finished; sums run
 * in a fixed order, so results repeat bit for bit. */

/* Inputs and targets of the learned warm start.  The network maps the reduced covariance of
 * one mode to the state that mode takes in the solved MPS; the warm start is the product state
 * of its predictions (vtn_mps_product), from which the sweeps begin instead of a random MPS.
 * Features of mode i from its 2 x 2 reduced covariance V_i (Eq. for the covariance; xxpp
 * blocks of V): [log V_xx, log V_pp, V_xp / sqrt(V_xx V_pp), log det V_i / 2] -> out
 * float[M*VTN_WARM_NFEAT].  Host only; VTN_EUNSUPPORTED for MPOs given as cores. */
#define VTN_WARM_NFEAT 4
vtn_status vtn_warm_features(vtn_mpo mpo, float* out);
/* Targets from a solved state: for every mode i the dominant eigenvector u_i of its reduced
 * density matrix (vtn_reduced_density; the mode's best single-mode state), phase fixed so that
 * u_i[0] is real and non-negative, as out float[M*2d] with (Re, Im) interleaved. */
vtn_status vtn_warm_targets(vtn_ctx ctx, vtn_mpo mpo, vtn_mps mps, float* out);

/* Create with He-uniform weights (W_l entries uniform in +-sqrt(6 / n_in_l) from a splitmix64
 * stream seeded with seed), zero biases and zero Adam moments.  1 <= n_in, width, n_out <= 4096,
 * 0 <= depth <= 16. */
vtn_status vtn_mlp_create(vtn_ctx ctx, int n_in, int width, int depth, int n_out, uint64_t seed, vtn_mlp* out);
vtn_status vtn_mlp_free(vtn_mlp mlp);
/* Shape, parameter count and Adam steps taken (each pointer may be NULL). */
vtn_status vtn_mlp_info(vtn_mlp mlp, int* n_in, int* width, int* depth, int* n_out, long long* n_params,
                        long long* steps);
/* Copy the parameters to / from host float[n_params]; set also clears the Adam moments and
 * the step count. */
vtn_status vtn_mlp_get_params(vtn_ctx ctx, vtn_mlp mlp, float* host);
vtn_status vtn_mlp_set_params(vtn_ctx ctx, vtn_mlp mlp, const float* host);
/* y = net(x) for batch rows (1 <= batch <= 4,000,000). */
vtn_status vtn_mlp_forward(vtn_ctx ctx, vtn_mlp mlp, int batch, const float* x, float* y);
/* loss = mean over batch*n_out entries of (net(x) - t)^2 (host float) and its gradient with
 * respect to the parameters (host float[n_params]; may be NULL). */
vtn_status vtn_mlp_loss_grad(vtn_ctx ctx, vtn_mlp mlp, int batch, const float* x, const float* t, float* loss,
                             float* grad);
/* One Adam step with learning rate lr > 0 on the batch; loss (host, may be NULL) is the loss
 * before the step. */
vtn_status vtn_mlp_train_step(vtn_ctx ctx, vtn_mlp mlp, int batch, const float* x, const float* t, float lr,
                              float* loss);

/* `steps` Adam steps (as vtn_mlp_train_step) on one batch without returning to the host in between;
 * loss (host, may be NULL) = the loss before the last step.  1 <= steps <= 1e7. */
vtn_status vtn_mlp_train(vtn_ctx ctx, vtn_mlp mlp, int batch, const float* x, const float* t, float lr, int steps,
                         float* loss);
/* The learned warm start of an instance: the network (n_in = VTN_WARM_NFEAT, n_out = 2 d) maps the
 * features of every mode (vtn_warm_features) to a site vector (2 d floats read as d complex
 * amplitudes), and the state is their product (vtn_mps_product); pass it to vtn_sweep as the
 * initial state.  VTN_EINVAL if the network's shape does not match; a prediction that is zero for
 * some mode is rejected like in vtn_mps_product. */
vtn_status vtn_mps_warm_start(vtn_ctx ctx, vtn_mpo mpo, vtn_mlp mlp, vtn_mps* out);

/* Real bf16 GEMM on the tensor cores (the kernel behind VTN_BF16X3):
 *   D[m][n] = sum_k A[m][k] * B[n][k], FP32 accumulation,
 * A: device bf16[M][lda], B: device bf16[N][ldb] (row-major, K contiguous, 16-byte aligned
 * base and row strides), K a positive multiple of 64; D: device float[M][ldd]
 * (d_fp64 = 0) or double[M][ldd] (d_fp64 != 0).  A library facility used by the solver's
 * split-precision products; exposed for parity tests and kernel timing. */
vtn_status vtn_gemm_bf16(vtn_ctx ctx, int M, int N, int K, const void* A, long long lda, const void* B,
                         long long ldb, void* D, long long ldd, int d_fp64);

/* Accumulation length of the split-precision tensor-core products: the largest number of
 * 64-wide k-blocks (bf16 split operands) one tensor-memory accumulator sums before its FP32
 * partial is added to the others by compensated FP32 summation (longer sums are split along k).  The tensor cores'
 * FP32 accumulation loses accuracy about linearly with the sum's length, so shorter runs are
 * more accurate and cost more split-K partial traffic.  env_kblocks applies to the environment
 * updates (vtn_env_update and those of the sweeps: their errors add up along the chain),
 * heff_kblocks to H_eff psi.  Defaults 64 and 256; each must be in [1, 4096].  Per context. */
vtn_status vtn_set_tc_accumulation(vtn_ctx ctx, int env_kblocks, int heff_kblocks);

/* Form of the truncation's Householder tridiagonalisation (one persistent cooperative kernel
 * either way): for n >= min_n the kernel keeps only the lower triangle of the trailing matrix up
 * to date (8 instead of 12 FP64 multiply-adds per element and column, two grid barriers per
 * column instead of one), below it the full matrix.  Default 1200 (measured, lower against full:
 * 207 against 270 ms at n = 3072, 81 against 94 at 2048, 46 against 49 at 1536, 23.6 against
 * 22.0 at 1024); 0 = always the lower form, above 4096 = never.  Per context; results agree to
 * rounding. */
vtn_status vtn_set_tridiag_lower(vtn_ctx ctx, int min_n);

/* Turn per-kernel device timing (CUDA events on the context stream) on or off and read
 * the accumulated figures: launches, algorithmic flops and seconds per kernel class.
 * classes: 0 = complex GEMM (all), 1 = GEMMs inside H_eff psi, 2 = truncation eigensolver,
 * 3 = Lanczos vector kernels, 4 = W mixing, 5 = tensor-core GEMMs (bf16 flops executed;
 * class 1 counts their useful complex flops), 6 = the Householder tridiagonalisation of the
 * truncation (16/3 n^3 real flops per n x n Hermitian matrix). */
vtn_status vtn_timing(vtn_ctx ctx, int enable);
vtn_status vtn_timing_read(vtn_ctx ctx, int cls, long long* launches, double* flops, double* seconds);
vtn_status vtn_timing_reset(vtn_ctx ctx);

#ifdef __cplusplus
}
#endif

#endif /* VTN_H */
