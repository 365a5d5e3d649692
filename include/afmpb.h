/*
 * afmpb.h -- C ABI of the GB300 node-patch Poisson-Boltzmann boundary-integral library.
 *
 * The library solves the linearized Poisson-Boltzmann equation (paper Sec. 2, Eq. 2) in
 * its second-kind boundary-integral form (Eq. 3), discretised by the node-patch scheme
 * (Eq. 4-6, Fig. 1):
 *
 *      [ alpha I + B      -A        ] [f]     1   [ sum_k q_k G(x_p, r_k)        ]
 *      [ D           alpha I - C    ] [h]  = ---- [ sum_k q_k dG/dn0(x_p, r_k)   ]     (Eq. 5)
 *                                           eps_out
 *
 * with alpha = 1/(2 eps_bar) + 1/2, eps_bar = eps_out / eps_in, G = 1/(4 pi r),
 * u = exp(-kappa r)/(4 pi r), f = exterior potential and h = its outward normal
 * derivative on the surface nodes.  A, B, C, D are the patch integrals of Eq. 6: near
 * pairs are integrated over the patch detail once at create time, far pairs use the
 * node values (integrand constant over the patch), and the far sums are evaluated with
 * an adaptive fast multipole method that carries the Laplace and Yukawa single- and
 * double-layer potentials and their normal derivatives in one tree pass (the four FMM
 * calls of the solution flow in Sec. 2, step 3b).  The linear system is solved by
 * restarted GMRES (Sec. 3.4) with the stop test of Eq. 7.
 *
 * Conventions
 *  - Every call returns an afmpb_status and never aborts.  On failure the handle's
 *    afmpb_last_error() string says why (thread-local string when the handle is NULL).
 *    Host failures inside the library (a host allocation or a host thread that could
 *    not be created) return AFMPB_ENOMEM; any other internal host failure returns
 *    AFMPB_EINTERNAL.  A create that fails frees whatever it had built.
 *  - Lengths are in Angstrom, charges in units of e, kappa in 1/Angstrom, energies in
 *    kcal/mol.
 *  - "Caller order" is the node order of the mesh passed to afmpb_create.  The
 *    unknown vector is x = [f; h] (length 2N), the product y = [y1; y2] (length 2N).
 *  - Host pointers are read during the call only; the library copies what it keeps.
 *    Device pointers must stay valid until the work queued on the handle's stream has
 *    completed.
 *  - A handle is not thread-safe.  Use one handle per host thread.
 *  - All GPU work of a handle runs on its stream (afmpb_options.stream, or a stream the
 *    handle creates when that field is NULL).  The handle owns all device memory it
 *    allocates until afmpb_destroy.
 */
#ifndef AFMPB_H
#define AFMPB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct afmpb_t afmpb_t;

typedef enum {
    AFMPB_OK = 0,
    AFMPB_EINVAL = 1,    /* invalid argument (NULL pointer, size, parameter range)   */
    AFMPB_EMESH = 2,     /* mesh not closed, not edge-manifold, mis-oriented,
                            degenerate triangle, or index out of range               */
    AFMPB_ENOMEM = 3,    /* device or host allocation failed                         */
    AFMPB_ECUDA = 4,     /* a CUDA runtime call failed (message has the CUDA error)  */
    AFMPB_ENOCONV = 5,   /* GMRES did not converge within max_restart; best iterate kept */
    AFMPB_ETIMEOUT = 6,  /* a bounded device wait expired                            */
    AFMPB_EBUSY = 7,     /* operation refused while other work owns the handle       */
    AFMPB_ESTATE = 8,    /* call out of order (e.g. energy before a successful solve) */
    AFMPB_EINTERNAL = 9  /* an internal numerical step failed (the eigensolver of the
                            M2L compression did not converge)                        */
} afmpb_status;

/* Surface mesh (host memory).  Triangles are counter-clockwise when seen from the
 * solvent, so that (b - a) x (c - a) points outward (Eq. 2: n points to the solvent). */
typedef struct {
    int64_t n_nodes;
    int64_t n_tris;
    const double *xyz;      /* [n_nodes * 3] node positions                          */
    const int32_t *tri;     /* [n_tris * 3] node indices, 0-based                     */
    const double *normals;  /* optional [n_nodes * 3] unit outward node normals; NULL =
                               normalised area-weighted mean of incident facet normals */
} afmpb_mesh;

/* Point charges of the molecule (host memory), Eq. 1-2: q_k at r_k. */
typedef struct {
    int64_t n;
    const double *xyz;      /* [n * 3] */
    const double *q;        /* [n]     */
} afmpb_charges;

/* afmpb_options.leaf_cap: choose the leaf capacity by measurement (afmpb_get_autotune). */
#define AFMPB_LEAF_CAP_AUTO (-1)

/* Options; a zero-initialised struct selects every default. */
typedef struct {
    int leaf_cap;        /* most nodes in a leaf box of the octree (default 80 with
                            precision 1, 192 with precision 0); AFMPB_LEAF_CAP_AUTO tunes it */
    int restart;         /* GMRES Krylov dimension m (default 80, Sec. 5)                */
    int max_restart;     /* GMRES restarts allowed (default 5, Sec. 5)                   */
    double abs_tol;      /* eps_abs of Eq. 7 (default 0)                                 */
    int precision;       /* 0 = FP32 FMM; 1 = mixed: M2L on the tensor cores (BF16 split
                            into three products, FP32 accumulation)                      */
    double near_c;       /* near-set factor c: t is near p when
                            |x_p - x_t| < c (rho_p + rho_t), rho = patch radius (default 2) */
    void *stream;        /* cudaStream_t to run on, or NULL                              */
    int max_level;       /* deepest octree level (default and maximum 20)                */
    double m2l_tol;      /* list-2 translations are compressed to the singular vectors of
                            the stacked translation matrices whose singular values exceed
                            m2l_tol times the largest (default 1e-5 for 0; a negative
                            value keeps the full n^3 x n^3 translations)                 */
    int charge_fmm;      /* charge-surface sums of the right-hand side and the energy:
                            0 = by FMM when n_nodes x n_charges > AFMPB_CHARGE_FMM_PAIRS,
                            else direct; 1 = always direct; 2 = always by FMM            */
    int orth;            /* Arnoldi orthogonalisation: 0 = classical Gram-Schmidt applied
                            twice (three reductions per step, default); 1 = one reduction per
                            step (AFMPB_ORTH_ONE_REDUCTION) */
    int m2l_method;      /* list-2 translations: 0 = dense (compressed, tensor cores with
                            precision 1; default); 1 = plane waves (AFMPB_M2L_PLANE_WAVE):
                            the exponential expansions of FMM97 (Sec. 3.1) in six directions,
                            quadratures accurate to 1e-6 of 1/r, FP32 CUDA cores            */
} afmpb_options;

#define AFMPB_M2L_PLANE_WAVE 1

/* afmpb_options.restart: no restart -- the Krylov dimension is the largest whose FP64
 * basis fits in half of the free device memory at the first solve (at most
 * AFMPB_RESTART_NONE_MAX); the paper's no-restart runs (Sec. 5). */
#define AFMPB_RESTART_NONE (-1)
#define AFMPB_RESTART_NONE_MAX 4096
/* afmpb_options.orth = 1: classical Gram-Schmidt with one fused reduction per Arnoldi step
 * (the coefficients V^T w and ||w||^2 together), ||w - V h|| from Pythagoras
 * (||w||^2 - ||h||^2), and a second Gram-Schmidt pass only when that norm falls below 1e-3
 * of ||w|| (loss of orthogonality; the reorthogonalisation test of the FP64 reference
 * GMRES).  The communication-hiding direction of the paper's future work (Sec. 6). */
#define AFMPB_ORTH_ONE_REDUCTION 1

/* afmpb_options.charge_fmm = 0 switches to the FMM above this many charge-node pairs. */
#define AFMPB_CHARGE_FMM_PAIRS 5.0e11

/* Solve report. */
typedef struct {
    int iters;             /* Arnoldi steps over all cycles                             */
    int restarts;          /* restart cycles after the first                            */
    double res_est;        /* final Givens residual estimate |g_{j+1}|                  */
    double res_true;       /* ||b - L x|| / ||b|| with one more product                 */
    double bnorm;          /* ||b||_2                                                    */
    double ms_setup;       /* time spent in afmpb_create (host clock)                   */
    double ms_matvec_total;/* time inside products during the solve: the number of
                              products times the CUDA-event time of the final one       */
    double ms_gmres;       /* time of the whole solve (CUDA events)                     */
    int64_t nnz_near;      /* stored near-field pairs (incl. the diagonal)              */
    int64_t n_boxes;       /* octree boxes                                               */
    int krylov_dim;        /* Krylov dimension m used (restart, or the no-restart size)  */
    int second_passes;     /* Arnoldi steps that took a second Gram-Schmidt pass (orth = 1;
                              every step with orth = 0)                                  */
} afmpb_solve_info;

/* Structure sizes (for tests, tooling and the memory estimator). */
typedef struct {
    int64_t n_nodes, n_tris, n_atoms;
    int64_t n_boxes, n_leaves, n_levels;
    int64_t nnz_near;
    int64_t n_list_u, n_list_v, n_list_w, n_list_x;   /* total entries of lists 1-4    */
    int64_t n_p2p_pairs;       /* sum over targets of their P2P sources (lists 1 and 3)  */
    int64_t n_m2l_pairs;       /* V-list (list 2) translations per product              */
    int order;                 /* Chebyshev points per dimension of each expansion      */
    int precision;
    int64_t device_bytes;      /* device memory held by the handle                     */
    double root_center[3];
    double root_half_width;
    double ms_create[6];       /* afmpb_create phases (host clock): geometry, tree and lists,
                                  near field, FMM operators, right-hand side, graph capture */
    int m2l_rank;              /* compressed translation size r (0: full n^3)            */
    int m2l_tables;            /* compressed bases: Laplace + one Yukawa per level       */
    int64_t device_bytes_peak; /* high-water mark of device_bytes (setup scratch included) */
    int leaf_cap;              /* leaf capacity the octree was built with                */
    int autotuned;             /* 1 when AFMPB_LEAF_CAP_AUTO ran the tuner for this handle */
    int charge_fmm;            /* 1 when the right-hand side and energy use the FMM      */
    int64_t charge_fmm_boxes;  /* boxes of that FMM's octree over nodes and charges      */
} afmpb_info;

/* Leaf-capacity and tile-shape autotuner report (AFMPB_LEAF_CAP_AUTO; no counterpart in
 * the paper, which fixes the leaf size by hand).  The handle is first built at start_cap; its product's
 * stage times calibrate the cost of one list-2 translation (ms_per_m2l_pair) and of one
 * box in the other tree passes (ms_per_box); for each candidate capacity the octree and
 * lists alone are rebuilt over the same geometry and the P2P kernel is timed on them
 * (p2p_ms); predicted_ms = p2p_ms + ms_per_m2l_pair * list-2 pairs + ms_per_box * boxes +
 * ms_rest.  The handle is rebuilt at best_cap when that predicts a product at least 3%
 * faster.  The choice is cached per size class (device, precision, order, kappa > 0,
 * floor(log2 N)), tile shapes included; later handles of the class start at it and skip
 * the tuning. */
#define AFMPB_AUTOTUNE_MAX 16
typedef struct {
    int n_candidates;
    int cap[AFMPB_AUTOTUNE_MAX];
    double p2p_ms[AFMPB_AUTOTUNE_MAX];
    double predicted_ms[AFMPB_AUTOTUNE_MAX];
    int start_cap, best_cap;
    double predicted_start_ms, predicted_best_ms;
    double ms_per_m2l_pair, ms_per_box, ms_rest;
    double ms_tuning;          /* host time of the calibration and the candidate trees   */
    /* Tile shapes, chosen on the handle built at best_cap by timing the kernels themselves:
     * P2P blocks kept resident per SM (4-6) x work units per block (1-6), and the number of
     * offsets per work item of the tensor-core M2L (8-32; 0 when that kernel is not used). */
    int p2p_resident, p2p_units_per_block, m2l_runs_per_item;
    double p2p_ms_default, p2p_ms_tuned;   /* P2P at the library defaults and at the choice  */
    double m2l_ms_default, m2l_ms_tuned;   /* the same for the M2L translations              */
} afmpb_autotune_report;

/* Per-stage timing of one product (afmpb_profile_product). */
#define AFMPB_MAX_STAGES 16
typedef struct {
    int n_stages;
    char name[AFMPB_MAX_STAGES][16];   /* "gather", "p2m", "m2m", "m2l", "p2l", "l2l", "l2p",
                                          "p2p", "combine", "scatter"                    */
    double ms[AFMPB_MAX_STAGES];       /* mean duration of the stage (CUDA events)        */
    int launches[AFMPB_MAX_STAGES];    /* kernel launches of the stage per product       */
    double ms_graph;                   /* mean duration of the captured product (graph)   */
    int kernels_per_product;           /* kernel launches of one afmpb_matvec call       */
} afmpb_profile;

/* Select parts of the product for testing (afmpb_matvec_parts). */
#define AFMPB_PART_DIAG 1  /* alpha x                                                 */
#define AFMPB_PART_FAR 2   /* point (far-rule) sums over every t != p: FMM + P2P     */
#define AFMPB_PART_NEAR 4  /* near correction: near rule minus far rule on N(p), plus
                              the self patch                                           */
#define AFMPB_PART_ALL 7

/* Build the handle: validate the mesh, compute node-patch geometry (Fig. 1), sort the
 * nodes along a Morton curve, build the adaptive octree and its four interaction lists
 * (Sec. 3.2: list 3 is evaluated point to point like list 1), integrate the near-field
 * patch coefficients of Eq. 6 once (Sec. 2, step 2), build the FMM operators, and, when
 * charges are given, the right-hand side of Eq. 5 (step 1).
 *   mesh       required; checked (EMESH on failure)
 *   charges    may be NULL (then afmpb_solve / afmpb_energy return ESTATE)
 *   eps_in, eps_out > 0; kappa >= 0; fmm_order in [2, 8] Chebyshev points per dimension;
 *   tol = eps_rel of Eq. 7 (> 0); options may be NULL.
 * On success *out receives the handle. */
afmpb_status afmpb_create(const afmpb_mesh *mesh, const afmpb_charges *charges,
                          double eps_in, double eps_out, double kappa, int fmm_order,
                          double tol, const afmpb_options *options, afmpb_t **out);

/* y = L x for the operator of Eq. 5 (caller order, device pointers, FP32, length 2N).
 * Queued on the handle's stream; returns before the product completes.  x and y must not
 * overlap.
 * Bounded waits: the tensor-core translation kernels (precision 1) give up on a device wait
 * after a fixed number of polls and set the handle's wait flag instead of hanging.  The
 * flag is latched: the next afmpb_matvec, afmpb_matvec_parts, afmpb_matvec_host or
 * afmpb_solve call on the handle, or afmpb_sync, returns AFMPB_ETIMEOUT once (queuing
 * nothing) and clears it; the products queued since the previous report are invalid. */
afmpb_status afmpb_matvec(afmpb_t *h, const float *x_dev, float *y_dev);

/* As afmpb_matvec but only the selected AFMPB_PART_* terms are summed into y. */
afmpb_status afmpb_matvec_parts(afmpb_t *h, const float *x_dev, float *y_dev, int parts);

/* Host-buffer product: copies x to the device, forms y = L x, copies y back and waits.
 * x_host, y_host: [2N] caller order.  Returns AFMPB_ETIMEOUT when a bounded device wait of
 * this product (or a latched one of an earlier product) expired; y is then invalid. */
afmpb_status afmpb_matvec_host(afmpb_t *h, const float *x_host, float *y_host);

/* Waits until the work queued on the handle's stream has finished.  Returns AFMPB_ETIMEOUT
 * (once, clearing the latched flag) when a bounded device wait of that work expired, ECUDA
 * when the stream reports an error, else OK. */
afmpb_status afmpb_sync(afmpb_t *h);

/* Fault injection for tests of the AFMPB_ETIMEOUT path (no counterpart in the paper): waits
 * for the handle's stream, then sets the handle's wait flag from the host exactly as an
 * expired device wait would.  No kernel runs and no device wait is made to expire. */
afmpb_status afmpb_inject_wait_expiry(afmpb_t *h);

/* Solve Eq. 5 with restarted GMRES on the device (FP64 basis, Arnoldi with classical
 * Gram-Schmidt applied twice or the one-reduction form of afmpb_options.orth, Givens
 * rotations, stop test of Eq. 7), starting from x = 0.  Each restart cycle runs on the
 * device as one graph launch: the Arnoldi steps form a graph WHILE loop whose last kernel
 * applies the stop test, so the host waits once per cycle, not once per step.
 * f_host / h_host ([N] each, caller order) may be NULL; the solution stays in the handle.
 * Returns ENOCONV when max_restart cycles did not reach the tolerance (the best iterate
 * is still stored and returned).  info may be NULL. */
afmpb_status afmpb_solve(afmpb_t *h, double *f_host, double *h_host, afmpb_solve_info *info);

/* Batched solve: k problems' GMRES in lockstep, with the products fused across them.
 * The paper solves one problem at a time (Sec. 5 times single runs) and points to
 * accelerators for the near field (Sec. 5, Sec. 6); running many small problems together
 * on one GPU is this library's serving form of that solve.
 * Each handle keeps its own tree, operators, Krylov basis (afmpb_options restart, orth,
 * max_restart, tol of its creation) and solution; every Arnoldi step of all running
 * problems is one pass of one device graph: one P2P launch over the union of their work
 * units (ordered by cost across problems), one target-stationary tensor-core M2L launch
 * over all their translation items (when every handle has precision 1 with the same
 * compressed rank; else each problem's M2L stays in its own chain), and each problem's
 * remaining product and orthogonalisation kernels on a branch of their own.  A problem
 * whose Givens residual meets Eq. 7 or whose basis is full stops taking part at once (a
 * device flag that its kernels and its share of the fused work check); a restart cycle of
 * the batch is one graph launch and the host waits once per cycle.  The arithmetic of
 * each problem is that of afmpb_solve; results differ from a lone solve only by the
 * order of floating-point atomic additions.
 *   hs          k distinct handles with charges, all on one device; 1 <= k <= AFMPB_BATCH_MAX
 *   f_host, h_host  NULL, or k pointers each NULL or [N_i] (caller order) receiving the
 *               surface solution of problem i
 *   infos       NULL or [k]; ms_gmres is the batch's wall time, the same for all
 *   statuses    NULL or [k]: OK, ENOCONV (max_restart cycles without the tolerance) or
 *               ETIMEOUT (a bounded device wait of the batch expired) per problem
 * Returns OK when every problem converged, else ENOCONV or ETIMEOUT as above, or EINVAL /
 * ESTATE / ENOMEM / ECUDA for the batch.  The handles must not be used by other threads
 * during the call. */
#define AFMPB_BATCH_MAX 64
afmpb_status afmpb_solve_batch(afmpb_t *const *hs, int k, double *const *f_host, double *const *h_host,
                               afmpb_solve_info *infos, afmpb_status *statuses);

/* Polar solvation energy (kcal/mol) of the last solution:
 * E = 1/2 sum_k q_k phi_reac(r_k), phi_reac from the interior Green representation of
 * the surface solution.  Requires a successful (or ENOCONV) afmpb_solve.  phi_reac is
 * summed directly, or, when the handle uses the charge FMM (afmpb_options.charge_fmm,
 * afmpb_info.charge_fmm), by a Laplace FMM over the nodes and the charges (~1e-5
 * relative to the direct sum). */
afmpb_status afmpb_energy(afmpb_t *h, double *kcal_per_mol);

/* Allocation-free variant of afmpb_energy, for callers that cannot call cudaMalloc:
 * processes whose device memory is fully reserved by another allocator (a framework
 * memory pool or a fixed serving budget), and latency-critical loops that cannot afford
 * the device-wide synchronisation an allocation or free can cause.  afmpb_energy
 * allocates its partial-sum buffers on every call; this variant instead uses one
 * scratch array compiled into the library as a static device array of
 * 16 x AFMPB_NOALLOC_MAX_ATOMS + AFMPB_NOALLOC_MAX_ATOMS + 1 doubles (about 8.4 MB),
 * which every GPU that loads the library holds until the process exits.
 *   h             a handle with a prior afmpb_solve (ESTATE otherwise)
 *   kcal_per_mol  host output, the same energy afmpb_energy returns
 * With direct charge sums the result equals afmpb_energy's bit for bit.  With the charge
 * FMM (afmpb_info.charge_fmm = 1) every evaluation of the reaction potential adds the
 * FMM's translated expansions with FP32 atomics in a varying order, so two evaluations, and
 * this call against afmpb_energy, agree to about 1e-6 relative, not bit for bit.
 * Returns EINVAL when the handle has more than AFMPB_NOALLOC_MAX_ATOMS charges, or when
 * the calling thread's current device is not the device the handle was created on.  The
 * first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and caches it; make that first call before any stream capture.  A cudaDeviceReset by
 * the caller invalidates the cached address: do not call this entry point after one.  All
 * calls on one device share the one array, so the library serialises them: a call holds a
 * process-wide lock from its first kernel until its result is back on the host.  The
 * paper has no counterpart to this entry point. */
#define AFMPB_NOALLOC_MAX_ATOMS 65536
afmpb_status afmpb_energy_noalloc(afmpb_t *h, double *kcal_per_mol);

/* The right-hand side of Eq. 5 (caller order, host [2N]), formed at create time directly
 * or by the charge FMM (afmpb_options.charge_fmm; ~1e-5 relative L2 per block). */
afmpb_status afmpb_rhs(afmpb_t *h, double *b_host);

/* Node-patch geometry in caller order (host buffers, each may be NULL): patch area [N],
 * node normal [N*3], patch radius rho [N]. */
afmpb_status afmpb_get_geometry(afmpb_t *h, double *area, double *normals, double *rho);

/* Near-field CSR in caller order.  rowptr [N+1]; col [nnz]; coef [nnz*4] holds
 * (dA, dB, dC, dD); whole [nnz] tells which of two values an entry holds.  whole = 0:
 * near rule minus far (point) rule -- the product's far part already holds the point
 * rule for that pair.  whole = 1: the whole near-rule value, for the self entry (the
 * self-patch integrals of Eq. 6) and for the close pairs that the point-to-point pass
 * leaves out (FP32 distance r <= 0.9 c (rho_p + rho_t), every one of them inside the
 * near set r < c (rho_p + rho_t)).  Columns of a row are in the octree's Morton order.
 * Pass NULLs to skip. */
afmpb_status afmpb_get_near(afmpb_t *h, int64_t *rowptr, int32_t *col, float *coef,
                            uint8_t *whole);

/* Octree export (host buffers sized from afmpb_get_info; any may be NULL):
 *   box_level [n_boxes], box_anchor [n_boxes*3] (integer cell coordinates at the box's
 *   level), box_range [n_boxes*2] (node range in Morton order), box_parent [n_boxes],
 *   perm [n_nodes] (Morton position -> caller index), and the lists as CSR over boxes:
 *   u/w point-to-point lists are indexed by box (empty for non-leaves), v and x by box.
 *   *_ptr arrays have n_boxes+1 entries. */
afmpb_status afmpb_get_tree(afmpb_t *h, int32_t *box_level, int32_t *box_anchor,
                            int32_t *box_range, int32_t *box_parent, int32_t *perm,
                            int64_t *u_ptr, int32_t *u_idx, int64_t *v_ptr, int32_t *v_idx,
                            int64_t *w_ptr, int32_t *w_idx, int64_t *x_ptr, int32_t *x_idx);

afmpb_status afmpb_get_info(const afmpb_t *h, afmpb_info *info);

/* The tuner's report; ESTATE when the handle was not built with AFMPB_LEAF_CAP_AUTO or its
 * size class was already tuned (then info.autotuned = 0). */
afmpb_status afmpb_get_autotune(const afmpb_t *h, afmpb_autotune_report *report);

/* Time the stages of the product on the handle's stream: reps products run stage by
 * stage (not as a graph, P2P serialised after the far field) with CUDA events between
 * stages, then reps graph replays.  Before each repetition, flush_bytes of flush_dev
 * (device memory, may be NULL) are overwritten to evict the L2 cache.  The input is the
 * handle's last product result (values do not change the timing); results go to scratch
 * buffers of the handle.  Blocks until done. */
afmpb_status afmpb_profile_product(afmpb_t *h, int reps, void *flush_dev, size_t flush_bytes,
                                   afmpb_profile *out);

afmpb_status afmpb_destroy(afmpb_t *h);

/* Last error message of the handle (or of this thread when h is NULL); never NULL. */
const char *afmpb_last_error(const afmpb_t *h);

/* Upper estimate of the device bytes afmpb_create + afmpb_solve will hold. */
size_t afmpb_estimate_bytes(int64_t n_nodes, int64_t n_atoms, int fmm_order,
                            const afmpb_options *options);

/* Library version string. */
const char *afmpb_version(void);

/* Self-test of the bounded device waits (no counterpart in the paper).  Every wait of the
 * library's kernels on an mbarrier gives up after a fixed number of polls, records an error
 * flag that the host turns into AFMPB_ETIMEOUT, and lets the kernel return, so that the
 * context stays usable.  This call runs that mechanism on purpose: one thread waits, with
 * at most spin_limit polls (1 .. 2^26), on a shared-memory mbarrier that nothing ever
 * arrives at, on the current device and its own stream.
 *   expired  host output: 1 when the wait gave up and the flag reached the host (the
 *            expected outcome), 0 otherwise
 * Returns EINVAL for a spin_limit out of range or a NULL expired, ECUDA on a launch or
 * copy failure, else OK. */
afmpb_status afmpb_selftest_bounded_wait(int spin_limit, int *expired);

/* ---- Serving: continuous batching of whole solves ------------------------------------
 * The paper runs one solve at a time; this layer (no counterpart in the paper) serves
 * many molecules or conformations of uneven size on one GPU.  Each request is one full
 * afmpb_create + afmpb_solve + afmpb_energy + afmpb_destroy.  The server owns max_slots
 * slot threads, each with its own CUDA stream; a slot admits the first queued request (in
 * arrival order) whose device-memory reservation, afmpb_estimate_bytes of the request,
 * fits under bytes_budget beside the requests already running; once the request's setup is
 * done its reservation drops to the handle's measured high-water mark or its current bytes
 * plus the GMRES basis still to come, whichever is larger.  Requests that arrive while
 * others run are admitted as soon as a slot and memory free up, and their kernels overlap
 * on the device.  The inputs are copied at submission; the solution, if asked for, is
 * written into caller buffers that must stay valid until the request completes.  A result
 * is handed out once (poll or wait); the ticket is invalid afterwards.  All calls are
 * thread-safe except afmpb_server_destroy, which must not race with other calls on the
 * same server: it drops queued requests, lets running ones finish and frees the server. */
typedef struct afmpb_server_t afmpb_server_t;

typedef struct {
    afmpb_mesh mesh;             /* as for afmpb_create; copied at submission             */
    afmpb_charges charges;       /* copied at submission                                  */
    double eps_in, eps_out, kappa;
    int fmm_order;
    double tol;
    afmpb_options options;       /* options.stream is ignored: each slot has its own       */
    double *f_out, *h_out;       /* optional host buffers [n_nodes] for f and h (caller
                                    order), written before the request completes           */
} afmpb_request;

typedef struct {
    afmpb_status status;         /* AFMPB_OK, or the status of the failing step           */
    char error[160];             /* its message                                           */
    double energy_kcal_mol;
    afmpb_solve_info info;
    double t_submit, t_admit, t_done;   /* seconds since afmpb_server_create (steady clock) */
    int64_t bytes_reserved;      /* admission reservation                                 */
    int64_t bytes_used;          /* the handle's device high-water mark                   */
    int slot;
} afmpb_result;

typedef struct {
    int64_t submitted, completed, failed, running, queued;
    int64_t bytes_in_use, bytes_high_water, bytes_budget;   /* reservations              */
    int64_t max_running;         /* most requests running at once so far                  */
    int slots;
    int max_batch;               /* batched servers: the largest batch solved so far      */
    int64_t batches;             /* batched servers: batched solves run                   */
    int64_t batched_requests;    /* batched servers: requests solved in them              */
} afmpb_server_info;

/* bytes_budget > 0; max_slots in [1, 256].  The server runs every request on the device
 * that is current in the calling thread. */
afmpb_status afmpb_server_create(size_t bytes_budget, int max_slots, afmpb_server_t **out);

/* As afmpb_server_create, with batched solves (max_batch in [1, AFMPB_BATCH_MAX]; 1 is
 * afmpb_server_create; solvers in [1, 256], used when max_batch > 1).  The max_slots
 * slots only set requests up (each handle on a stream of its own); each of the solver
 * threads takes the oldest set-up request together with the other set-up requests of
 * similar size (node counts within a factor of two), up to max_batch, and solves them
 * with afmpb_solve_batch: their GMRES steps share fused P2P and M2L launches.  Requests
 * set up while solves run form the next batches.  Admission, reservations and results
 * are as for afmpb_server_create; a result's slot is the slot that set it up. */
afmpb_status afmpb_server_create_batched(size_t bytes_budget, int max_slots, int solvers, int max_batch,
                                         afmpb_server_t **out);
/* EINVAL for missing arrays or sizes; ENOMEM when the reservation exceeds the whole budget
 * (the request could never run); otherwise queues it and returns its ticket. */
afmpb_status afmpb_server_submit(afmpb_server_t *s, const afmpb_request *req, int64_t *ticket);
/* OK with *res filled when the request has completed (successfully or not), EBUSY while it
 * is queued or running, EINVAL for an unknown ticket. */
afmpb_status afmpb_server_poll(afmpb_server_t *s, int64_t ticket, afmpb_result *res);
/* As poll but blocks up to timeout_s seconds (>= 1e6 or infinity: no limit); ETIMEOUT if
 * the request is still pending, EINVAL if the ticket is unknown or another thread took
 * its result meanwhile. */
afmpb_status afmpb_server_wait(afmpb_server_t *s, int64_t ticket, double timeout_s, afmpb_result *res);
afmpb_status afmpb_server_get_info(afmpb_server_t *s, afmpb_server_info *st);
afmpb_status afmpb_server_destroy(afmpb_server_t *s);

/* ---- One solve on several GPUs: the partition plan --------------------------------------
 * The paper distributes one solve over many nodes (Sec. 3.3-3.4): the surface nodes, and
 * with them the rows of the product and every Krylov vector, are split along the Morton
 * order.  Each rank evaluates the rows of its nodes and needs from the others (a) the
 * unknowns (f, h) of the source nodes outside its range that its point-to-point pairs
 * (lists 1 and 3, list 4) and its near-field rows read -- the halo, exchanged before each
 * product; (b) the multipole expansions of list-2 source boxes it does not own (a box whose
 * nodes lie on several ranks is shared: its expansion is the sum of the ranks' partial
 * ones); (c) global sums of the Krylov inner products.  This host-only call computes (a)
 * and (b) from the arrays afmpb_get_tree and afmpb_get_near export, with the node ranges
 * cut between leaves so that the ranks' estimated work (targets x point-to-point sources +
 * near-field entries) is balanced.  No GPU is touched.  (The multi-GPU product kernels are
 * not part of this library: every GB300 machine here has one GPU.) */
typedef struct {
    int64_t n_nodes, n_boxes;
    const int32_t *box_range;    /* [n_boxes*2] node range in Morton order (a box's range
                                    covers its subtree)                                   */
    const int32_t *box_parent;   /* [n_boxes], -1 for the root                            */
    const int64_t *u_ptr; const int32_t *u_idx;   /* lists 1-4 as CSR over boxes, as     */
    const int64_t *v_ptr; const int32_t *v_idx;   /* afmpb_get_tree exports them         */
    const int64_t *w_ptr; const int32_t *w_idx;
    const int64_t *x_ptr; const int32_t *x_idx;
    const int64_t *near_ptr;     /* optional [n_nodes+1] near-field rows in Morton order   */
    const int32_t *near_col;     /* their columns (Morton positions); NULL with near_ptr   */
} afmpb_plan_input;

typedef struct {
    int64_t node_begin, node_end;  /* the rank's Morton range of nodes (rows)             */
    int64_t n_halo;                /* nodes of other ranks whose unknowns it reads        */
    int64_t n_send;                /* (node, destination) pairs of its own nodes others read */
    int64_t n_import_boxes;        /* list-2 source boxes whose expansion it receives     */
    int64_t n_shared_boxes;        /* boxes touching its range whose nodes span ranks     */
    double work;                   /* its work estimate                                   */
} afmpb_plan_rank;

typedef struct afmpb_plan_t afmpb_plan_t;
/* EINVAL for a NULL array, nranks < 1 or a box range / parent out of bounds. */
afmpb_status afmpb_plan_create(const afmpb_plan_input *in, int nranks, afmpb_plan_t **out);
afmpb_status afmpb_plan_get_rank(const afmpb_plan_t *p, int rank, afmpb_plan_rank *info);
/* halo nodes [n_halo] (ascending) and the rank owning each */
afmpb_status afmpb_plan_get_halo(const afmpb_plan_t *p, int rank, int64_t *nodes, int32_t *owner);
/* own nodes sent [n_send] and their destination ranks, grouped by destination */
afmpb_status afmpb_plan_get_send(const afmpb_plan_t *p, int rank, int64_t *nodes, int32_t *dest);
/* imported boxes [n_import_boxes] with their owner (-1: shared), shared boxes [n_shared_boxes] */
afmpb_status afmpb_plan_get_boxes(const afmpb_plan_t *p, int rank, int32_t *imports, int32_t *import_owner,
                                  int32_t *shared);
afmpb_status afmpb_plan_destroy(afmpb_plan_t *p);

#ifdef __cplusplus
}
#endif

#endif /* AFMPB_H */
