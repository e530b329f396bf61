/*
 * tns.h -- C ABI of the GB300 two-site DMRG H_eff*psi engine.
 *
 * The engine implements the projected superblock product of two-site DMRG for
 * the general long-range Hamiltonian of Eq. (1) (Sec. III) under U(1)xU(1)
 * symmetry (particle number n, 2*S_z).  With the two dots' local spaces split
 * into one-dimensional sectors, H_eff*psi reduces to a sum of products
 * B += alpha * sum_i L_i A R_i^T (Eq. 2), one per symmetry block and per
 * left/right operator pair; the operators come from normal/complementary
 * operator partial summation (Sec. III.A.2, "Independent operational tasks").
 *
 * Conventions
 *  - All functions return TNS_OK (0) or a negative TNS_ERR_* code; nothing
 *    aborts or throws across the ABI.  tns_last_error() describes the last
 *    failure of a context.
 *  - Orbitals 0..N-1, spin-orbital p = 2*i + s (s = 0 up, 1 down), Jordan-
 *    Wigner order (0up, 0dn, 1up, ...).  Site basis |0>,|up>,|dn>,|updn> with
 *    |updn> = c+_up c+_dn |0>.  Quantum number (n, two_sz) = (0,0),(1,1),
 *    (1,-1),(2,0) per site state.
 *  - Bond b (0..N) is labelled by the quantum numbers of orbitals 0..b-1
 *    ("left counted").
 *  - Host pointers are read during the call and never retained; the caller
 *    keeps ownership.  Device pointers passed to tns_heff_apply are owned by
 *    the caller and must stay valid until the call's work on the context's
 *    stream has finished (all entry points synchronise the stream before
 *    returning, except where stated).
 *  - One context is bound to one CUDA device and one stream; a context must
 *    not be used from two host threads at once.
 */
#ifndef TNS_H
#define TNS_H

#ifdef __cplusplus
extern "C" {
#endif

#define TNS_OK 0
#define TNS_ERR_ARG (-1)            /* invalid argument (size, index, symmetry of v, ...) */
#define TNS_ERR_STATE (-2)          /* call made out of order */
#define TNS_ERR_OOM (-3)            /* device (or host) allocation failed */
#define TNS_ERR_NOCONV (-4)         /* Davidson did not reach the tolerance; best estimate kept */
#define TNS_ERR_DEVICE_TIMEOUT (-5) /* a bounded device wait gave up; context stays usable */
#define TNS_ERR_CUDA (-6)           /* a CUDA runtime call failed */

/* arithmetic of the sector GEMMs in tns_heff_apply */
#define TNS_FP64 0    /* native FP64 (DFMA) */
#define TNS_TF32 1    /* TF32 operands, FP32 accumulation (tcgen05 kind::tf32; mma.sync m16n8k8 for blocks <= 32) */
#define TNS_BF16X3 2  /* split-BF16 hi/lo, 3 products, FP32 accumulation (tcgen05 kind::f16; mma.sync m16n8k16) */

typedef struct tns_ctx tns_ctx;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (NULL: the context creates and owns a non-blocking stream).  *out is set on
 * success. */
int tns_create(tns_ctx** out, int device, void* cuda_stream);

/* Release every device and host resource of the context.  NULL is ignored. */
void tns_destroy(tns_ctx* ctx);

/* Text of the last error of this context ("" if none).  Valid until the next
 * call on the same context. */
const char* tns_last_error(const tns_ctx* ctx);

/* Integrals of Eq. (1) (Sec. III): h[i*N+j] = h_ij (symmetric) and
 * v[((i*N+j)*N+k)*N+l] = (ij|kl) in chemist order with the 8-fold symmetry;
 * e_core is added to every energy.  Both arrays are host, row-major, copied.
 * Returns TNS_ERR_ARG if N < 2, N > 128, h is not symmetric or v breaks the
 * 8-fold symmetry by more than 1e-12 (absolute). */
int tns_load_integrals(tns_ctx* ctx, int N, const double* h, const double* v, double e_core);

/* Initial MPS in the (n_elec, two_sz) sector with bond dimension at most D
 * (D sets the accuracy, Sec. III).  Every bond gets all symmetry sectors the
 * sector can reach, with dims bounded by the Schmidt rank and scaled to D;
 * site tensors are 0/1 right-canonical isometries (each right basis state is a
 * distinct determinant), chosen with a seed-driven counter-based shuffle.
 * Requires tns_load_integrals.  TNS_ERR_ARG for an unreachable sector. */
int tns_mps_init(tns_ctx* ctx, int N, int n_elec, int two_sz, int D, unsigned long long seed);

/* Replace the MPS by a caller-given one (import / restart).  First
 * tns_mps_define(N, n_elec, two_sz, D); then, for every bond b in 0..N,
 * tns_mps_set_bond(b, nsec, sectors, dims) with sectors = nsec (n, two_sz)
 * pairs (left counted, strictly increasing by (n, two_sz)) and dims = nsec
 * positive dimensions; then, for every site b in 0..N-1, tns_mps_set_site(b,
 * blocks, len) where `blocks` concatenates, for each bond-b sector q_l in bond
 * order and each site state s = 0..3 whose q_l+qn(s) is a bond-(b+1) sector,
 * the dim(q_l) x dim(q_l+qn(s)) row-major block (len = total doubles).
 * Site tensors left of the two-site step used must be left-canonical and
 * those right of it right-canonical for H_eff to be the projected
 * Hamiltonian; the arithmetic of tns_build_env / tns_heff_apply does not
 * depend on it.  tns_mps_get_site copies the same layout back to the host
 * (len must equal the size; pass blocks=NULL to query it in *len_out). */
int tns_mps_define(tns_ctx* ctx, int N, int n_elec, int two_sz, int D);
int tns_mps_set_bond(tns_ctx* ctx, int bond, int nsec, const int* sectors, const int* dims);
int tns_mps_set_site(tns_ctx* ctx, int site, const double* blocks, long long len);
int tns_mps_get_bond(tns_ctx* ctx, int bond, int* nsec, int* sectors, int* dims, int cap);
int tns_mps_get_site(tns_ctx* ctx, int site, double* blocks, long long len, long long* len_out);

/* Build the left block of orbitals 0..site-1 and the right block of orbitals
 * site+2..N-1 (blocking + renormalisation, Sec. III; complementary operator
 * partial sums, Sec. III.A.2), then the operator table x task table of the
 * two-site step (site, site+1) (Sec. III.A.2: operator-table rows, task-table
 * rows, position index).  Blocks already built for the current MPS are
 * reused.  0 <= site <= N-2. */
int tns_build_env(tns_ctx* ctx, int site);

/* Layout of the two-site wavefunction at step (site, site+1), valid after
 * tns_build_env(site): its symmetry blocks, the first level of the task
 * hierarchy of Sec. III.A.1 (the quantum-number sectors that split the
 * superblock vector into independent dense blocks).  *desc points to n_blocks rows of 9 int64 values
 * (n_l, two_sz_l, s1, s2, n_r, two_sz_r, m, n, offset): q_l = (n_l, two_sz_l)
 * is a bond-`site` sector (left counted), q_r = (n_r, two_sz_r) the particle
 * content of orbitals site+2..N-1, the block is m x n row-major at element
 * `offset` of a vector of *length doubles.  Blocks are ordered by (q_l in
 * bond order, s1, s2, q_r).  The pointer stays valid until the next
 * tns_build_env or MPS change. */
int tns_psi_layout(tns_ctx* ctx, int site, int* n_blocks, const long long** desc, long long* length);

/* Y = H_eff X at step (site, site+1) (Eq. 2 summed over all operator pairs and
 * symmetry blocks; Alg. 2 computes the same sums).  X and Y are DEVICE
 * pointers to nvec vectors of `length` doubles each (vector j at offset
 * j*length), in the layout of tns_psi_layout; they must not overlap.  Y is
 * overwritten.  precision: TNS_FP64, TNS_TF32 or TNS_BF16X3 (the latter two
 * run the sector products on tensor cores with FP32 accumulation: tcgen05
 * tiles for output blocks above 32 states, warp-level tiles for output blocks
 * whose dimensions and those of all X blocks they read are at most 32 -- the
 * limit is the environment variable TNS_TC_SMALL read when the context is
 * created).  Requires tns_build_env(site).  Runs on the context stream and
 * synchronises it. */
int tns_heff_apply(tns_ctx* ctx, int site, const double* X, double* Y, int nvec, int precision);

/* One part of an operator-row split of tns_heff_apply (Sec. "Independent
 * operational tasks": the rows of the operator table -- the pairs of normal
 * and complementary operators -- are distributed over devices, every device
 * accumulates the output blocks of its rows, and one sum over the devices
 * gives H_eff X).  The rows are assigned to nparts parts by their flop cost
 * (longest first onto the least loaded part); the assignment depends only on
 * the step, so every caller with the same MPS and integrals gets the same
 * split.  Y (DEVICE, nvec vectors of `length`) is overwritten with the sum over
 * the rows of part `part` (0 <= part < nparts); summing Y over all parts (e.g.
 * an all-reduce across ranks) gives tns_heff_apply's result up to rounding
 * order.  Same arguments, layout and precisions as tns_heff_apply. */
int tns_heff_apply_part(tns_ctx* ctx, int site, const double* X, double* Y, int nvec, int precision, int part,
                        int nparts);

/* Diagonal of H_eff at step (site, site+1) into the DEVICE vector diag
 * (length doubles).  Used as the Davidson preconditioner. */
int tns_heff_diag(tns_ctx* ctx, int site, double* diag);

/* Differentiation form (not in the paper; adjoint of Eq. 2).  The operator
 * catalogues of the left block (orbitals 0..site-1, side 0) and of the right
 * block (orbitals site+2..N-1, side 1) used by step (site, site+1) live in one
 * DEVICE arena each; tns_env_arena returns its pointer and length (doubles).
 * The arena may be modified by the caller (e.g. to perturb an operator); call
 * tns_build_env(site) afterwards so the partial sums are recomputed.  The
 * operators of an empty block (the left block of step 0, the right block of
 * step N-2) are zero by definition and are never read.
 * Layout: operators in catalogue order, each operator its symmetry blocks
 * (out <- in) row-major. */
int tns_env_arena(tns_ctx* ctx, int site, int side, double** data, long long* size);

/* Adjoint of Y = H_eff X at step (site, site+1) for the cotangent Ybar:
 * Xbar = H_eff^T Ybar (= H_eff Ybar, H_eff being symmetric), and the gradients
 * of <Ybar, H_eff X> with respect to every element of the left and right
 * arenas of tns_env_arena: per product alpha L X R^T the contributions
 * alpha Ybar R X^T (to L) and alpha Ybar^T L X (to R), carried through the
 * partial sums to the catalogue operators.  All pointers are DEVICE; X, Ybar,
 * Xbar have the layout of tns_psi_layout, Lbar/Rbar the arena lengths; any of
 * Xbar, Lbar, Rbar may be NULL.  Outputs are overwritten.  FP64. */
int tns_heff_adjoint(tns_ctx* ctx, int site, const double* X, const double* Ybar, double* Xbar, double* Lbar,
                     double* Rbar);

/* Allocation-free variant of tns_heff_diag (the paper has no counterpart;
 * this is a service to callers).  Callers that must not allocate device
 * memory at this point -- code running under a memory pool that reserves
 * the whole device, or inside a region where a cudaMalloc would synchronise
 * the device or fail with out-of-memory -- cannot use tns_heff_diag, which
 * uploads its per-call index tables into freshly allocated buffers.  This
 * entry point stages them instead into one fixed file-scope device array of
 * TNS_NOALLOC_DIAG_MAX int entries (16 MiB), which every GPU that loads the
 * library holds until the process exits, and calls no cudaMalloc, cudaFree
 * or allocating library routine.
 *  - Same arguments and result as tns_heff_diag (diag: DEVICE, length doubles,
 *    fully overwritten).
 *  - Requires the step's work list to be resident on the device already: call
 *    tns_heff_apply or tns_heff_diag once for this step first; otherwise
 *    TNS_ERR_STATE.
 *  - TNS_ERR_ARG if the step's diagonal work list needs more than
 *    TNS_NOALLOC_DIAG_MAX index entries.
 *  - The first call on a device looks up the array's device address (once
 *    per device and CUDA context, with that device current: again after a
 *    device reset); make that first call before any stream capture.
 *  - All calls share the array and each call rewrites the part it uses, so
 *    nothing carries over between calls; calls that overlap on the GPU (from
 *    several contexts or threads) race on it and must be serialised. */
#define TNS_NOALLOC_DIAG_MAX (4 * 1024 * 1024)
int tns_heff_diag_noalloc(tns_ctx* ctx, int site, double* diag);

/* Lowest eigenpair of H_eff at step (site, site+1) by block Davidson on the
 * device (FP64 orthogonalisation, Rayleigh quotient and residual).  X is a
 * DEVICE vector of `length` doubles: on entry the start vector (zero vector:
 * a default start is used), on exit the normalised eigenvector.  *energy
 * receives the eigenvalue + e_core, *iters the number of matrix-vector
 * products.  precision as in tns_heff_apply; reduced precisions are
 * corrected with FP64 residuals.  TNS_ERR_NOCONV if tol is not reached in
 * max_iter products (X and *energy hold the best estimate). */
int tns_davidson(tns_ctx* ctx, int site, double* X, double tol, int max_iter, int precision,
                 double* energy, int* iters);

/* Differentiation form, integral gradients (not in the paper): dE/dh and
 * dE/dv of E = <psi|H_eff|psi> / <psi|psi> at step (site, site+1) with the
 * MPS isometries fixed -- by Hellmann-Feynman the 1- and 2-particle reduced
 * density matrices of the state the MPS and psi represent, for the
 * Hamiltonian of Eq. (1) written as sum h_ij E_ij + 1/2 sum (ij|kl) e_ijkl.
 * Computed by reverse mode through the products of Eq. (2) and through the
 * renormalisation chain (blocking, rotation, partial sums) of both blocks
 * down to the empty blocks.
 *  - psi: DEVICE, layout of tns_psi_layout(site), need not be normalised.
 *  - gamma: HOST N*N, gamma[i*N+j] = dE/dh_ij symmetrised over (i, j)
 *    = sum_s <a+_is a_js>.
 *  - Gamma: HOST N^4 or NULL, Gamma[((i*N+j)*N+k)*N+l] = 2 dE/d(ij|kl)
 *    averaged over the eight index permutations that leave (ij|kl)
 *    unchanged (only these orbit sums are defined for integrals with the
 *    8-fold symmetry) = the orbit average of sum_st <a+_is a+_kt a_lt a_js>.
 * Requires tns_build_env(site).  FP64.  Synchronous. */
int tns_rdm(tns_ctx* ctx, int site, const double* psi, double* gamma, double* Gamma);

/* Batched dense symmetric eigen-decomposition, the solver the truncation uses
 * on each middle-bond sector's reduced density matrix (the SVD hand-off of the
 * two-site step, Sec. III.A; Householder tridiagonalisation then implicit QR
 * with the Wilkinson shift, one CTA per matrix).  nmat matrices of sizes n[i]
 * (HOST array, each n[i] <= 4096) packed one after another, row-major, in the
 * DEVICE array A (sum n[i]^2 doubles; overwritten).  Z (DEVICE, same size)
 * receives eigenvector p of matrix i as row p of its n[i] x n[i] block; w
 * (DEVICE, sum n[i] doubles) the eigenvalues, unsorted, in the same order.
 * Synchronous.  TNS_ERR_ARG for a size above the limit, TNS_ERR_NOCONV if a
 * matrix hits the QR step limit. */
int tns_sym_eig(tns_ctx* ctx, int nmat, const int* n, double* A, double* Z, double* w);

typedef struct tns_sweep_opts {
  int nsweeps;         /* full sweeps (left->right then right->left) */
  int D;                /* bond dimension cap (<= the D of the MPS) */
  double tol;           /* Davidson residual tolerance (2-norm, normalised vector) */
  int max_iter;         /* Davidson matrix-vector products per step */
  int precision;        /* TNS_FP64 / TNS_TF32 / TNS_BF16X3 */
  double cutoff;        /* singular values <= cutoff are dropped (e.g. 1e-14) */
  int verbose;          /* print one line per step on stdout */
  int block;            /* Davidson block size: corrections from the lowest `block`
                           Ritz pairs per iteration, their products in one
                           batched H_eff*psi launch; 0 or 1 = single vector, max 4 */
} tns_sweep_opts;

typedef struct tns_sweep_stats {
  double energy;            /* lowest energy seen in the last sweep (incl. e_core) */
  double max_discarded;     /* largest discarded weight of the last sweep */
  long long matvecs;        /* H_eff*psi products over the whole call */
  double heff_flops;        /* useful FP64-equivalent flops of those products */
  double heff_seconds;      /* device time inside H_eff*psi */
  double env_seconds;       /* device time of environment builds */
  double svd_seconds;       /* device time of truncations */
  double seconds;           /* wall time of the call */
  int steps;                /* two-site steps done */
  int max_bond;             /* largest bond dimension after the call */
} tns_sweep_stats;

/* Two-site DMRG sweeps over the current MPS (tns_mps_init or an import),
 * the sweep of Sec. III / Sec. IV.A (a sweep is one left-to-right and one
 * right-to-left pass of two-site iteration cycles; D sets the accuracy):
 * per step environment build, Davidson on H_eff, SVD truncation to at most D
 * states, renormalisation.  *energy_out receives the final energy.  stats is
 * optional (NULL). */
int tns_sweep(tns_ctx* ctx, const tns_sweep_opts* opts, double* energy_out, tns_sweep_stats* stats);

typedef struct tns_step_stats {
  double energy;            /* Davidson eigenvalue (incl. e_core) */
  double discarded;         /* discarded weight of the truncation */
  int iters;                /* H_eff*psi products of the step */
  int converged;            /* 1 if the Davidson tolerance was reached */
  double heff_flops;        /* useful FP64-equivalent flops of those products */
  double heff_seconds;      /* device time inside H_eff*psi (CUDA events on the context stream) */
  double env_seconds;       /* partial sums, work lists and renormalisation */
  double svd_seconds;       /* truncation */
  double seconds;           /* wall time of the call */
  long long length;         /* two-site wavefunction length */
  int bond_dim;             /* new dimension of bond site+1 */
  long long kernel_launches; /* launches of the engine's own CUDA kernels in the call */
  int exact_products;       /* FP64 products among iters (reduced-precision refreshes; 0 on the FP64 path) */
  double exact_seconds;     /* device time of those FP64 products */
  double env_flops;         /* FP64 flops of the step's renormalisation products */
  double env_bytes;         /* algorithmic bytes of the step's partial sums and renormalisation
                               (operands read once, results written once) */
} tns_step_stats;

/* One two-site step of a sweep at (site, site+1) (one "DMRG iteration cycle",
 * Sec. IV.A): environment (reused if current), Davidson on H_eff, truncation
 * at bond site+1 to at most opts->D states, and renormalisation of the
 * block that grows (left block if left_to_right, else right block).
 * x0_host: optional HOST start vector in the layout of tns_psi_layout(site)
 * (NULL: the two-site product of the current site tensors); psi_host:
 * optional HOST output of the converged two-site wavefunction (same layout).
 * Both are copied synchronously inside the call.  opts->nsweeps is ignored.
 * Returns TNS_OK also when Davidson stops at max_iter (stats->converged = 0). */
int tns_step(tns_ctx* ctx, int site, int left_to_right, const tns_sweep_opts* opts, const double* x0_host,
             double* psi_host, tns_step_stats* stats);

/* Two-site product of the current site tensors at (site, site+1) in the layout
 * of tns_psi_layout(site) (the default Davidson start of tns_step), copied to
 * the HOST array x_host; *length receives its length (x_host NULL: length
 * only).  Works without tns_build_env. */
int tns_psi_guess(tns_ctx* ctx, int site, double* x_host, long long* length);

/* Useful FP64-equivalent flop count of one tns_heff_apply(site) for nvec = 1
 * (the per-product cost of Eq. (2) with the cheaper chain order of Sec. III.B):
 * one product per operator pair of the expansion, per pair of dot blocks
 * (s1' <- s1, s2' <- s2) and per X symmetry block, costing min(2mr(n+q),
 * 2qn(m+r)) for the m x n X block, q x m left and r x n right operator blocks;
 * a factor that is a multiple of the block identity costs nothing (2mnr,
 * 2qmn, or 2mn when both are); products whose operator block is identically
 * zero are not counted.  *nproducts receives the number of block products the
 * kernels execute (each expression of a dot block is one product there). */
int tns_heff_flops(tns_ctx* ctx, int site, double* flops, long long* nproducts);

/* Checkpoint / restart of a sweep (the long FeMoco runs of Sec. "Model
 * systems" restart from a stored MPS).  tns_checkpoint_save writes the
 * integrals, the MPS (bond sectors and site tensors) and a sweep position
 * (the next step's site and direction, stored as given) to the file `path`
 * (binary, little-endian, versioned, ended by a 64-bit FNV-1a hash of its
 * contents).  tns_checkpoint_load reads such a file into the context,
 * replacing its integrals and MPS (environments are rebuilt on demand), and
 * returns the position (site, left_to_right may be NULL).  A file that is
 * not a checkpoint, truncated or altered is refused with TNS_ERR_ARG before
 * the context changes.  Synchronous. */
int tns_checkpoint_save(tns_ctx* ctx, const char* path, int site, int left_to_right);
int tns_checkpoint_load(tns_ctx* ctx, const char* path, int* site, int* left_to_right);

/* Schedules of the grouped product (the batched form's autotuner): each new
 * work list of a precision and vector count first runs its schedule
 * variants in turn (split-K targets of 1, 2 and 4 rounds over the SMs; for the
 * tensor-core forms also the persistent warp-specialised kernel), timed with
 * CUDA events, and keeps the fastest; the choice is cached under a shape
 * signature of the list (product and block counts, histogram of output-block
 * sizes), so later lists of the same shape take it without tuning.
 * runs[p][v]: steady-state products of precision p (TNS_FP64, TNS_TF32,
 * TNS_BF16X3) that ran variant v. */
typedef struct tns_sched_stats {
  long long tuned;       /* work lists tuned */
  long long cache_hits;  /* work lists that took a cached choice */
  long long runs[3][4];
} tns_sched_stats;
int tns_schedule_stats(tns_ctx* ctx, tns_sched_stats* out);

/* Out-of-HBM environments (the tree-traversal cache of Alg. 1, Sec. "Tree-
 * Traversal Optimized Virtual Memory Addressing", applied to the chain of
 * left and right blocks).  The operator catalogues of all blocks of a sweep
 * grow as D^2 N^2 each; the engine keeps on the device the two that the
 * current step reads and moves the others off it when the device runs short:
 * in stack order (the catalogue needed last leaves first), to pinned host
 * memory while host_bytes last, else dropped and rebuilt from its neighbours
 * when the sweep needs it again.  Every step first makes a memory plan (its
 * partial sums, work list, tensor-core operand images and Davidson vectors)
 * and fails with TNS_ERR_OOM, before it allocates or launches anything, if
 * the plan does not fit next to its two catalogues.
 *  - device_bytes: most device memory the library may hold on the context's
 *    device (all contexts on that device share it); 0 = the device's size.
 *  - host_bytes: pinned host memory for staged catalogues; 0 = no staging
 *    (catalogues that must leave the device are dropped).
 * Results do not depend on either setting. */
int tns_set_memory_budget(tns_ctx* ctx, long long device_bytes, long long host_bytes);

typedef struct tns_mem_stats {
  long long device_used;   /* bytes the library holds on the device now */
  long long device_peak;   /* high-water mark since the last reset (reset=1 below) */
  long long device_limit;  /* the budget, else the device's size */
  long long host_used;     /* pinned host bytes holding staged catalogues */
  long long host_peak;
  long long staged;        /* catalogues moved to host memory */
  long long restored;      /* catalogues moved back to the device */
  long long dropped;       /* catalogues freed (rebuilt when needed) */
  long long built;         /* catalogues built by renormalisation */
  long long last_plan;     /* bytes of the last step's memory plan (beyond its catalogues) */
} tns_mem_stats;

/* Memory statistics of the context's device; reset != 0 restarts the
 * device high-water mark at the current use. */
int tns_memory_stats(tns_ctx* ctx, tns_mem_stats* out, int reset);

#ifdef __cplusplus
}
#endif
#endif /* TNS_H */
