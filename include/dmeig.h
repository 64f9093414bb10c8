/*
 * dmeig.h -- C ABI of the GB300 Dey--Mittra cavity eigensolver.
 *
 * Computes resonant modes of a perfectly conducting cavity on a Yee grid with
 * Dey--Mittra cut cells (Bauer, Werner & Cary, arXiv:1301.3794): the magnetic
 * eigenmodes b and wavenumbers k^2 of  A^-1 C L C^T b = k^2 b  (Sec. 2,
 * Eq. discWaveBDM), found by a shift-and-invert Krylov eigensolver on
 *     P_DM (K - sigma A)^-1 A,   K = C L C^T + A D^T V^-1 D A     (Eq. fullMat)
 * whose inner solves are flexible GMRES preconditioned by geometric multigrid.
 *
 * Conventions shared by every call:
 *  - Grid: nx, ny, nz cells of size dx, dy, dz; node (i,j,k) at
 *    origin + (i dx, j dy, k dz).  The outer walls are perfect conductors.
 *  - Level set phi at the (nx+1)(ny+1)(nz+1) nodes, i fastest (C order of an
 *    array shaped [nz+1][ny+1][nx+1]); phi < 0 is vacuum, phi >= 0 conductor.
 *  - Natural face layout ("F" doubles): x-faces [nz][ny][nx+1], then y-faces
 *    [nz][ny+1][nx], then z-faces [nz+1][ny][nx], each i fastest.  x-face
 *    (i,j,k) sits at x = x_i and spans [y_j, y_j+1] x [z_k, z_k+1].  Closed
 *    faces (area fraction 0) always hold 0.
 *  - Natural edge layout ("E" doubles): x-edges [nz+1][ny+1][nx], y-edges
 *    [nz+1][ny][nx+1], z-edges [nz][ny+1][nx+1].  Cells: [nz][ny][nx].
 *  - Pointers marked "host or device" are device pointers when the matching
 *    on_device flag is nonzero, host pointers otherwise.  The caller owns
 *    every buffer it passes; the library never keeps a caller pointer after a
 *    call returns.  The library owns its handles and their device workspaces.
 *  - All work is issued on the context's stream; calls return after that
 *    stream has finished the call's work.
 *  - No exception crosses the ABI.  On failure a call returns a nonzero
 *    dm_status and dm_last_error() describes the cause.
 */
#ifndef DMEIG_H
#define DMEIG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dm_status {
    DM_OK = 0,
    DM_ERR_INVALID_ARG = 1,
    DM_ERR_NO_CONVERGENCE = 2,
    DM_ERR_TIMEOUT = 3,
    DM_ERR_CUDA = 4,
    DM_ERR_OOM = 5,
    DM_ERR_GEOMETRY = 6
} dm_status;

/* Storage precision of the multigrid preconditioner (Krylov work stays FP64). */
typedef enum dm_precision {
    DM_PREC_F64 = 0,
    DM_PREC_F32 = 1,      /* FP32 storage and arithmetic */
    DM_PREC_BF16 = 2      /* BF16 vectors, FP32 coefficients and accumulation */
} dm_precision;

typedef struct dm_context dm_context;
typedef struct dm_geometry dm_geometry;
typedef struct dm_operator dm_operator;
typedef struct dm_learned dm_learned;

/* Multigrid preconditioner settings (a design of this library: the paper used
 * an algebraic V-cycle with one order-1 polynomial smoother step per level and
 * direction, Sec. 6). */
typedef struct dm_mg_params {
    int max_coarse;        /* halve the grid while every dim is even, >= 4, and max dim > max_coarse (4),
                              and while the level has more than dense_coarse open faces */
    int band_sweeps;       /* Jacobi sweeps of the cut-cell band smoother after each smoothing step on the
                              fine level (24; the coarser levels take band_sweeps_coarse):
                              a restricted additive Schwarz step over bricks of band_brick^3 nodes with
                              one node of overlap; each subdomain sweeps on its own faces, couplings to
                              other faces frozen, and the brick keeps the faces it owns */
    int band_brick;        /* brick edge in nodes (8); 0 < band_brick, and the largest subdomain must fit
                              the sweep buffers in shared memory (DM_ERR_INVALID_ARG otherwise) */
    double omega_scale;    /* Jacobi weight = omega_scale / lambda_max(D^-1 (K - sigma A)), and
                              omega_scale / 2 in the scalar cycle of P_DM (1.7) */
    int power_iters;       /* power iterations for lambda_max of the vector cycle (30); the scalar cycle
                              uses the bound 2 of D^-1 D A D^T (its rows sum to zero) */
    int precision;         /* dm_precision of the V-cycle (DM_PREC_F64) */
    int autotune;          /* 1: time the stencil tile shapes per level at setup and keep the fastest;
                              results are cached in the context by level size and precision (1) */
    int stencil_shape;     /* -1: the autotuner's choice (shape 0 when autotune = 0); 0..5: use this
                              tile shape (see dm_operator_stencil_shape) on every level (-1) */
    int band_sweeps_coarse; /* band_sweeps of the levels below the fine one (16) */
    int symmetric_transform; /* 1: the V-cycle of Eq. fullMat2's symmetric form (Sec. 5.3): every level
                              congruence-scaled by A^-1/2, which for this cycle amounts to the transfers
                              A_c^1/2 R A^-1/2 and A^-1/2 P A_c^1/2 (smoothing and the coarsest solve
                              are invariant under the scaling); the outer solves still use K (0) */
    int dense_coarse;      /* a level with at most this many open faces is the coarsest and is solved
                              densely (2048; 0 = coarsen by max_coarse alone; at most 6000) */
    int krylov_ff;         /* 1: inside the shifted solves' FGMRES iterations, (K - sigma A) z is formed in
                              float-float arithmetic (two FP32 numbers per value, about 48 significant
                              bits) on the FP32 pipes, straight into the float-float Krylov basis, and so
                              is D A D^T z inside the projection's scalar iterations; the restart
                              residuals, the final residual checks and every certificate stay in FP64.
                              0: the FP64 applies plus a gather.  Allocates about 72 bytes per fine-level
                              node on the geometry (1) */
    int jacobi_sweeps;     /* damped Jacobi sweeps of each smoothing step, before the band smoother, on
                              every level, pre and post (2; at most 16) */
} dm_mg_params;

typedef struct dm_eig_params {
    double sigma;          /* shift (Eq. shiftInv): modes with k^2 nearest sigma are found */
    int nev;               /* number of eigenpairs wanted */
    double tol;            /* Ritz residual tolerance, relative to |theta| (1e-10) */
    double inner_tol;      /* relative residual of each shifted solve (1e-9; the pairs are certified against
                              rho_tol whatever it is, see rho_tol) */
    double proj_tol;       /* scalar-solve tolerance inside P_DM, see dm_operator_project (1e-12) */
    int basis;             /* Krylov-Schur basis size m; 0 = max(2 nev + 10, 24) capped at 64 */
    int max_restarts;      /* (100) */
    int inner_restart;     /* FGMRES basis size (40) */
    int inner_maxit;       /* FGMRES iteration cap per solve (400) */
    unsigned long long seed; /* start vector seed */
    dm_mg_params mg;
    const dm_learned* learned; /* nullable: learned correction after each V-cycle (see dm_learned_*) */
    double max_seconds;    /* wall-clock limit of one eigensolve, setup included; 0 = none (0).  Checked
                              before every shifted solve: a solve that runs out returns DM_ERR_TIMEOUT */
    double rho_tol;        /* certificate every returned pair must meet, rho = ||K b - k^2 A b|| /
                              (k^2 ||A b||) in FP64 (1e-8; 0 = Ritz estimates only).  When the Ritz
                              estimates call the nev pairs converged but a certificate misses rho_tol,
                              the Ritz tolerance drops to a tenth of the worst current estimate, inner_tol
                              to a tenth (down to 1e-15 and 1e-13), and the Krylov-Schur basis is rebuilt
                              from the sum of the wanted Ritz vectors (a counted restart) */
} dm_eig_params;

typedef struct dm_eig_report {
    int n_converged;       /* leading eigenpairs (nearest sigma first) that met tol and rho_tol */
    int outer_iters;       /* Krylov-Schur expansion steps (= shifted solves) */
    int restarts;
    int inner_iters;       /* FGMRES iterations summed over all shifted solves */
    int proj_iters;        /* scalar FGMRES iterations summed over all projections */
    int mg_levels;
    double mg_complexity;  /* sum of open faces over levels / open faces of level 0 */
    double rho_max;        /* max ||K b - k^2 A b|| / (k^2 ||A b||) over returned pairs */
    double delta_max;      /* max ||D A b|| h / ||A b|| over returned pairs */
    double setup_seconds;  /* operator setup (diagonals, weights, coarsest factorisation) */
    double solve_seconds;  /* eigensolver iterations and certification */
    long long kernel_launches;  /* kernels this library launched during the call */
    int learned_applied;   /* preconditioner applications that used the learned correction */
    int learned_fallbacks; /* shifted solves in which it was switched off (residual stalled) */
} dm_eig_report;

/* ---- context ------------------------------------------------------------ */

/* Bind to CUDA device `device`; `cuda_stream` (a cudaStream_t, may be NULL)
 * is used for all work, NULL makes the library create its own stream. */
dm_status dm_context_create(int device, void* cuda_stream, dm_context** out);
/* Every geometry, operator and network made on `ctx` must be destroyed first:
 * their destroy functions synchronise the context's stream. */
void dm_context_destroy(dm_context* ctx);
/* Text of the last error on this context ("" if none).  Owned by the context. */
const char* dm_last_error(const dm_context* ctx);
/* Kernels launched on this context so far. */
long long dm_context_launch_count(const dm_context* ctx);
/* Device buffers, pinned host buffers, CUDA events, streams and graph
 * instantiations the library has created in this process, on any context (a
 * diagnostic with no counterpart in the paper: it lets a caller check that a
 * call which promises not to allocate, such as dm_operator_apply_noalloc,
 * created none).  Thread-safe. */
long long dm_debug_allocation_count(void);

/* ---- kernel timing (profiling aid; no counterpart in the paper) ---------- */
/* on = 1 clears the statistics and brackets every later kernel launch with a
 * pair of CUDA events on the context's stream; on = 0 stops recording. */
dm_status dm_trace_enable(dm_context* ctx, int on);
/* Number of distinct kernels timed so far (resolves pending events). */
int dm_trace_count(dm_context* ctx);
/* Entry i: kernel name (copied into name[name_cap]), launches, summed device ms. */
dm_status dm_trace_entry(dm_context* ctx, int i, char* name, int name_cap, long long* launches, double* total_ms);
/* Entry i: algorithmic DRAM bytes of its launches, summed, by the library's
 * per-kernel model (the bytes a launch must read and write at least, counted
 * on the elements that can be nonzero: open faces, band rows, active cells,
 * compact Krylov vectors); 0 for kernels without a model. */
dm_status dm_trace_entry_bytes(dm_context* ctx, int i, double* bytes);
/* FMA issue rates of the context's device, in TFLOP/s (2 flops per FMA), from
 * a register-resident loop of independent FMA chains timed with CUDA events
 * (best of 3 after a warm-up launch; about 0.1 s).  They are the peaks the
 * ALU-bound kernels (the FP64 operator apply) are measured against.  Either
 * pointer may be NULL. */
dm_status dm_measure_fma_rates(dm_context* ctx, double* fp64_tflops, double* fp32_tflops);

/* ---- geometry (Sec. 2, Eq. farInt / Fig. dmFace; Sec. 5.1, Eq. divBInt /
 *      Fig. dmVol; Sec. 6.1 tetrahedral cut volumes) ------------------------ */

/* Cut fractions L (edges), A (faces), V (cells) = parts *outside* the
 * conductor of the zero set of the piecewise-linear interpolant of phi on the
 * 6-tetrahedron (Kuhn) split of every cell; the multigrid levels' fractions
 * are averages of the fine ones.  phi: host or device, (nx+1)(ny+1)(nz+1).
 * a_min > 0 neglects faces with A < a_min and their edges (Sec. 3); 0 keeps
 * all faces (the paper's method).  nx, ny, nz >= 2.  A phi holding NaN or
 * infinite values is rejected with DM_ERR_GEOMETRY. */
dm_status dm_geometry_create(dm_context* ctx, int nx, int ny, int nz,
                             double dx, double dy, double dz, const double origin[3],
                             const double* phi, int phi_on_device, double a_min,
                             dm_geometry** out);
/* Kinds of the six outer walls (Sec. 6.2-6.3: symmetry planes that reduce the
 * domain).  DM_WALL_PEC: a perfect electric conductor on the wall's node plane
 * (normal faces and tangential edges closed); an electric symmetry plane is
 * this wall.  DM_WALL_PMC: a magnetic symmetry plane half a cell OUTSIDE the
 * wall's node plane (through the centres of the cells the mirror would add),
 * so the grid's first node plane lies h/2 from the plane; the wall's normal
 * faces and tangential edges keep their fractions and the field beyond is
 * zero.  With that placement the half-domain problem has exactly the modes of
 * the mirrored full domain whose normal flux is even under the mirror. */
typedef enum { DM_WALL_PEC = 0, DM_WALL_PMC = 1 } dm_wall;

/* dm_geometry_create with chosen wall kinds: walls[6] in the order x-low,
 * x-high, y-low, y-high, z-low, z-high (NULL = all DM_WALL_PEC).  The coarser
 * levels average the fine fractions, walls included.  A vacuum region that
 * reaches a magnetic wall carries no constant null vector of D A D^T (the
 * potential is zero beyond the wall), so P_DM pins nothing there.  An entry
 * that is neither kind gives DM_ERR_INVALID_ARG. */
dm_status dm_geometry_create_walls(dm_context* ctx, int nx, int ny, int nz, double dx, double dy, double dz,
                                   const double origin[3], const double* phi, int phi_on_device, double a_min,
                                   const int walls[6], dm_geometry** out);

/* A geometry from cut fractions the caller supplies instead of a level set:
 * L (edges, natural edge layout), A (faces) and V (cells), host or device per
 * on_device; the coarser multigrid levels average them as in
 * dm_geometry_create.  L and A must lie in [0, 1]; V must be finite and
 * non-negative and may exceed 1 (perturbed volumes, as in Sec. 6.1's study of
 * Eq. volPert1).  Entries on the outer walls are ignored: the walls are perfect
 * conductors.  Out-of-range values give DM_ERR_GEOMETRY. */
dm_status dm_geometry_create_from_fractions(dm_context* ctx, int nx, int ny, int nz, double dx, double dy, double dz,
                                            const double* L, const double* A, const double* V, int on_device,
                                            dm_geometry** out);
void dm_geometry_destroy(dm_geometry* geom);

/* Multigrid levels available below (and including) the fine grid. */
int dm_geometry_num_levels(const dm_geometry* geom);
/* dims[3] = cells of `level`; counts[4] = natural faces F, edges E, cells, open faces.
 * Counts are kept from the geometry's creation: the call launches nothing. */
dm_status dm_geometry_level_info(const dm_geometry* geom, int level, int dims[3], long long counts[4]);
/* Copy the fractions of `level` out in natural layouts: L (E), A (F), V (cells).
 * Any pointer may be NULL.  Host or device per on_device. */
dm_status dm_geometry_fractions(const dm_geometry* geom, int level, double* L, double* A,
                                double* V, int on_device);

/* ---- shifted operator and its preconditioner ----------------------------- */

void dm_mg_params_default(dm_mg_params* p);

/* K - sigma A (Eq. discLaplDM) on every level, with the V-cycle set up. */
dm_status dm_operator_create(dm_context* ctx, const dm_geometry* geom, double sigma,
                             const dm_mg_params* mg, dm_operator** out);
void dm_operator_destroy(dm_operator* op);
int dm_operator_num_levels(const dm_operator* op);
/* Tile shape the vector stencil of `level` uses: 0 = 32x4x2, 1 = 32x2x4, 2 = 32x8x1 nodes, one
 * node per thread; 3 = 32x8x8, 4 = 32x4x8, 5 = 32x8x4 nodes, a 32 x SY block marching along z
 * (chosen by the autotuner), -1 on a bad argument.  No counterpart in the paper. */
int dm_operator_stencil_shape(const dm_operator* op, int level);
/* Jacobi weight of `level` for the vector (scalar = 0) or the scalar (scalar = 1) cycle. */
double dm_operator_get_omega(const dm_operator* op, int level, int scalar);
dm_status dm_operator_set_omega(dm_operator* op, int level, int scalar, double omega);

/* y = (K - sigma A) x on `level` in FP64 (Eq. discLaplDM; K = C L C^T +
 * A D^T V^-1 D A with V^-1 = 0 where V = 0).  x, y: natural face layout. */
dm_status dm_operator_apply(dm_operator* op, int level, const double* x, double* y, int on_device);
/* The same product on the fine level as the shifted solves' FGMRES iterations
 * form it with krylov_ff = 1: float-float arithmetic (about 48 significant
 * bits), each open face's value hi + lo returned as an FP64 number (closed
 * faces 0).  DM_ERR_INVALID_ARG when the operator was created with
 * krylov_ff = 0.  x, y: natural face layout, caller-owned. */
dm_status dm_operator_apply_ff(dm_operator* op, const double* x, double* y, int on_device);
/* The same y = (K - sigma A) x as dm_operator_apply, for callers that must not
 * allocate memory once they are running: a loop that may not pay the device-
 * wide synchronisation cudaMalloc / cudaFree can cause, or an application
 * whose device memory is owned by its own pool allocator and capped, where an
 * extra cudaMalloc can fail or fragment the pool.  This call makes no device
 * or host allocation (no cudaMalloc, cudaFree, event or library allocator).
 * The paper has no counterpart; it is a service of this library.
 *  - x, y: device pointers, natural face layout of `level`.
 *  - Scratch: a static device array of 6,291,456 doubles (48 MiB) inside the
 *    library, held by every GPU that loads the library until the process exits.
 *    A call needs 6 * np doubles (np = padded node count of the level: about
 *    1.0 M nodes, i.e. grids up to roughly 100^3); larger levels are rejected
 *    with DM_ERR_INVALID_ARG and an explanatory dm_last_error().
 *  - The first call on each device looks up the scratch's device address
 *    (cudaGetSymbolAddress) with that device current.
 *  - Every call shares the one scratch array: calls that overlap on the GPU
 *    (other threads, other contexts or streams) race and corrupt each other's
 *    results; serialise them. */
dm_status dm_operator_apply_noalloc(dm_operator* op, int level, const double* x, double* y);
/* Diagonal of K - sigma A on `level` (natural face layout, 0 on closed faces). */
dm_status dm_operator_diagonal(dm_operator* op, int level, double* d, int on_device);
/* One smoothing step on `level` in the preconditioner's precision:
 * jacobi_sweeps times x <- x + omega D^-1 (f - (K - sigma A) x), then the band smoother (band_sweeps
 * sweeps per subdomain on the cut-cell band, see dm_mg_params).  x is updated
 * in place. */
dm_status dm_operator_smooth(dm_operator* op, int level, const double* f, double* x, int on_device);
/* f_c = R r = P^T r / 8 from `level` to level+1 (precision of the preconditioner). */
dm_status dm_operator_restrict(dm_operator* op, int level, const double* r, double* fc, int on_device);
/* x <- x + mask P e_c from level+1 to `level`. */
dm_status dm_operator_prolong(dm_operator* op, int level, const double* ec, double* x, int on_device);
/* e = one V(1,1) cycle applied to f on the fine level, from a zero guess. */
dm_status dm_operator_vcycle(dm_operator* op, const double* f, double* e, int on_device);
/* Solve (K - sigma A) x = b on the fine level by right-preconditioned FGMRES
 * to relative residual tol (Sec. 6: GMRES + multigrid).  x: output. */
dm_status dm_operator_solve(dm_operator* op, const double* b, double* x, int on_device,
                            double tol, int restart, int maxit, int* iters, double* relres);
/* y = P_DM x = x - D^T (D A D^T)^-1 D A x (Eq. proj); the scalar Laplacian is
 * solved by FGMRES + cell multigrid until its residual is below
 * tol * max(||D A x||, ||x|| / h_min): for a nearly divergence-free x the
 * divergence is rounding noise and only the field's own scale is meaningful. */
dm_status dm_operator_project(dm_operator* op, const double* x, double* y, int on_device,
                              double tol, int* iters);
/* One scalar V-cycle e ~= (D A D^T)^-1 f on cells (natural cell layout). */
dm_status dm_operator_scalar_vcycle(dm_operator* op, const double* f, double* e, int on_device);

/* ---- eigensolver (Sec. 4.1 Eq. shiftInv, Sec. 5.2 Eq. fullMat) ----------- */

void dm_eig_params_default(dm_eig_params* p);

/* The nev eigenpairs of A^-1 C L C^T b = k^2 b nearest sigma among the
 * electromagnetic (D A b = 0) modes, by Krylov-Schur on P_DM (K - sigma A)^-1 A
 * in the A inner product (Eq. bInner).  k2_out[nev] ascending (host).
 * b_out (nullable): nev x F, natural face layout, A-normalised (b^T A b = 1),
 * sign such that the entry of largest magnitude is positive; host or device
 * per b_on_device (a host b_out in page-locked memory is written by DMA at
 * link speed, pageable memory through the driver's staging).
 * DM_ERR_NO_CONVERGENCE still fills the converged prefix
 * and report->n_converged.  Two failures return no pair at all (k2_out set to
 * NaN, b_out untouched, n_converged = 0, the report's iteration counts and
 * timings filled):
 *  - the scalar solve inside P_DM reached its iteration cap (400) in 3
 *    projections of this eigensolve: DM_ERR_NO_CONVERGENCE, because without
 *    the projection the pairs cannot be trusted; the solve stops right after
 *    the third such projection;
 *  - p->max_seconds > 0 ran out before a shifted solve: DM_ERR_TIMEOUT. */
dm_status dm_eigensolve(dm_context* ctx, const dm_geometry* geom, const dm_eig_params* p,
                        double* k2_out, double* b_out, int b_on_device, dm_eig_report* report);

/* ---- learned smoother (no counterpart in the paper) -----------------------
 * A 3-layer 3x3x3 convolutional network without biases on the fine node grid
 * (8 -> 16 -> 16 -> 3 channels, relu between layers; BF16 activations, FP32
 * weights and accumulation).  Input per node: the residual on the node's x, y,
 * z faces divided by its RMS over the open faces, A_x, A_y, A_z, the node
 * cell's V, and 0.  Output: the error on those faces in units of RMS(r) h^2
 * (h = smallest spacing).  Inside the preconditioner it corrects the V-cycle
 * result z: with r = f - (K - sigma A) z and c the network's correction for r,
 * z <- z + alpha c where alpha = <r, K c> / <K c, K c> minimises the residual
 * along c (no step when alpha <= 0); the FP64 FGMRES residual decides on it and
 * switches it off for the rest of a solve when an iteration contracts by less
 * than 0.8.
 * Weights: [W1 | W2 | W3], each W[a][b][c][cin][cout] (a along k, b along j,
 * c along i), FP32. */
dm_status dm_learned_create(dm_context* ctx, unsigned long long seed, dm_learned** out);
void dm_learned_destroy(dm_learned* net);
long long dm_learned_num_params(void);
dm_status dm_learned_get_weights(const dm_learned* net, float* w);        /* host */
dm_status dm_learned_set_weights(dm_learned* net, const float* w);        /* host */
/* y = RMS(r) h^2 N(r / RMS(r), A, V) on the open faces of the geometry's fine grid
 * (natural face layouts, host or device per on_device). */
dm_status dm_learned_apply(dm_learned* net, const dm_geometry* geom, const double* r, double* y, int on_device);
/* Masked MSE 0.5 sum_open (Y - E)^2 / #open and its gradient for explicit
 * features X [(nz+1)(ny+1)(nx+1)][8] and targets E [...][3] (host, node order
 * i fastest, channel last).  grad: host, dm_learned_num_params() floats. */
dm_status dm_learned_loss_grad(dm_learned* net, const dm_geometry* geom, const float* X, const float* E, float* loss,
                               float* grad);
/* Train with Adam on the residuals the operator's plain V-cycle leaves: `runs`
 * seeded random right-hand sides, 8 Krylov directions each.  The objective is
 * the residual the correction leaves, 0.5 |r / RMS(r) - (K - sigma A) h^2 N(r)|^2
 * over the open faces / #open faces, with the operator in FP32 (its gradient is
 * K applied to that residual, K being symmetric).  loss_history (nullable,
 * host, epochs floats) receives the mean loss of every epoch. */
dm_status dm_learned_train(dm_learned* net, dm_operator* op, int runs, int epochs, float lr, unsigned long long seed,
                           float* loss_history);
/* One Adam step of the training above on a given residual r (natural face
 * layout, host or device per on_device; zero on closed faces): features from
 * r / RMS(r), the residual objective with op's operator in FP32, its gradient
 * by the backward pass, then the Adam update with step size lr (Adam's moment
 * state and step count carry over between calls; dm_learned_set_weights
 * resets them).  loss (nullable, host): the objective before the update;
 * grad (nullable, host, dm_learned_num_params() floats): its gradient. */
dm_status dm_learned_train_step(dm_learned* net, dm_operator* op, const double* r, int on_device, float lr,
                                float* loss, float* grad);
/* Use (net) or stop using (NULL) the learned correction in op's preconditioner.
 * In each shifted solve the FP64 FGMRES residual decides: an iteration that
 * contracts by less than 0.8 switches the correction off for the rest of that
 * solve, and after 3 solves in a row that switched it off the operator stops
 * offering it until this call sets a network again. */
dm_status dm_operator_set_learned(dm_operator* op, const dm_learned* net);

/* ---- batched eigensolves (many cavities and shifts; no counterpart in the paper) */

/* One work item: a cavity (geometry) with one shift and mode count.  k2_out
 * [params.nev] is host memory; b_out (nullable) is params.nev x F of that
 * cavity, host or device per b_on_device.  report and status are outputs. */
typedef struct dm_batch_item {
    const dm_geometry* geom;
    dm_eig_params params;
    double* k2_out;
    double* b_out;
    int b_on_device;
    dm_eig_report report;
    int status;
} dm_batch_item;

/* Solve every item; `streams` worker streams (>= 1) take items largest-first,
 * so the kernels of small cavities overlap on the GPU.  Each item's result is
 * the same as dm_eigensolve on it.  Returns DM_OK when every item returned
 * DM_OK, else the first non-OK item status (all items are still attempted).
 * Before the workers start, the stencil tile shapes of every distinct grid not
 * yet in the context's autotuner cache are timed on the calling stream with
 * the GPU otherwise idle (an operator setup per such grid).
 * Geometries must not be destroyed or shared with other calls meanwhile. */
dm_status dm_eigensolve_batched(dm_context* ctx, int n, dm_batch_item* items, int streams);

/* Residual certificate of n given eigenpairs (b: n x F natural layout):
 * rho = ||K b - k2 A b|| / (k2 ||A b||), delta = ||D A b|| h / ||A b||,
 * rq = b^T K b / b^T A b.  Outputs are host arrays of length n (nullable). */
dm_status dm_certify(dm_context* ctx, const dm_geometry* geom, int n, const double* k2,
                     const double* b, int on_device, double* rho, double* delta, double* rq);

#ifdef __cplusplus
}
#endif
#endif /* DMEIG_H */
