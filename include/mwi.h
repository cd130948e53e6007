/*
 * mwi.h -- C ABI of the GB300 microwave-imaging solver (libmwi.so).
 *
 * The library computes, on one GPU, the hot path of the paper's inversion
 * (Tournier et al., "Microwave Tomographic Imaging of Cerebrovascular
 * Accidents by Using High-Performance Computing"):
 *
 *   1. the time-harmonic curl-curl Maxwell problem (Section 2, Eq. pbdirect)
 *      discretised by Nedelec edge elements of degree 1 or 2 (Section 2.1),
 *      giving one linear system A u_j = b_j per transmitting antenna, all with
 *      the same complex-symmetric A (Eq. linsys);
 *   2. its solution by right-preconditioned flexible GMRES with the one-level
 *      ORAS preconditioner M^-1 = sum_i R_i^T D_i B_i^-1 R_i (Section 3,
 *      Eq. ORAS), all subdomains factorised and applied as one batch;
 *   3. the S-parameters (Section 4, Eq. sij), the misfit J (Section 5,
 *      Eq. defJ), the adjoint problem (Eq. pbadj) solved with the same
 *      operator and factors, and the per-tetrahedron gradient dJ/d eps_r.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Complex numbers are interleaved (re, im) pairs of double.
 * - Time factor exp(+i omega t): lossy media have Im(eps_r) < 0.  The
 *   factorisation runs without pivoting and relies on Im(A) being positive
 *   definite, which holds when every tet has Im(eps_r) < 0 (the LDL^T of a
 *   complex-symmetric matrix with positive-definite imaginary part exists).
 *   A pivot that still falls below a tiny threshold is perturbed and
 *   reported through mwi_solve_info.n_perturbed; FGMRES absorbs it.
 * - Ownership: every input array is caller-owned and copied (or read) during
 *   the call; every output array is caller-allocated.  Handles own all of
 *   their device memory.
 * - Errors: no C++ exception or abort crosses this boundary.  Every entry
 *   point returns an mwi_status; on a non-OK status mwi_last_error() returns
 *   a thread-local, human-readable message.  MWI_ENOTCONV still fills the
 *   outputs and the info struct.
 * - Streams: a problem's device work is ordered on the CUDA stream given to
 *   mwi_assemble (0 = the legacy default stream).  Calls return after that
 *   work has completed.  One handle must be used by one host thread at a time.
 * - Arrays marked "device" are device pointers on the current CUDA device;
 *   all others are host pointers.
 */
#ifndef MWI_H
#define MWI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MWI_OK = 0,
    MWI_EINVAL = 1,     /* bad argument (size, pointer, value) */
    MWI_ENOMEM = 2,     /* host or device allocation failed */
    MWI_ENOTCONV = 3,   /* FGMRES hit max_iter before rtol on some column */
    MWI_ECUDA = 4,      /* a CUDA runtime call failed */
    MWI_ETIMEOUT = 5,   /* reserved: bounded wait expired */
    MWI_ESTATE = 6,     /* call out of order (e.g. gradient before forward) */
    MWI_ESINGULAR = 7   /* a zero pivot could not be perturbed */
} mwi_status;

typedef struct mwi_mesh* mwi_mesh_t;       /* opaque: topology, DOFs, element geometry */
typedef struct mwi_problem* mwi_problem_t; /* opaque: A, ORAS factors, resident fields */

/* Edge-current dipole antenna (the paper's waveguide ports are replaced by a
 * current I on one mesh edge): the edge starts at the mesh vertex nearest to
 * pos and is the edge at that vertex best aligned with dir (ties: lowest
 * vertex id, then lowest edge id in (low, high) vertex-id order). */
typedef struct {
    double pos[3];
    double dir[3];
    double re_I, im_I;
} mwi_antenna;

/* Solver options.  Zero-initialised fields take the defaults in brackets. */
typedef struct {
    double rtol;          /* outer FGMRES relative residual, true ||b - A u|| / ||b|| [1e-6] */
    int32_t max_iter;     /* outer iterations per column, hard limit [500] */
    int32_t restart;      /* outer FGMRES restart length [50] */
    int32_t n_sub;        /* ORAS subdomains N_S [64] */
    int32_t overlap;      /* overlap delta in vertex-adjacent tet layers [1]; < 0 means none */
    int32_t precision;    /* 0 = complex FP64 everywhere;
                             1 = MIXED: complex FP32 subdomain factors and ORAS application as
                                 the preconditioner of the FP64 FGMRES (Arnoldi, residuals,
                                 least squares in FP64);
                             2 = MIXED_NESTED: an inner complex FP32 GMRES(ORAS) as the flexible
                                 preconditioner of the FP64 FGMRES [0] */
    int32_t inner_iters;  /* MIXED_NESTED: inner GMRES iterations per outer step [30] */
    double inner_rtol;    /* MIXED_NESTED: inner relative residual target [1e-4] */
    int32_t nd_leaf;      /* nested-dissection leaf size of the subdomain ordering [128] */
    int32_t verbose;      /* 0 silent, 1 phase timings on stderr [0] */
    const int32_t* part;  /* optional [nt] host array: caller's tet -> subdomain map
                             (values in [0, n_sub)); NULL = recursive coordinate bisection */
    int32_t max_block;    /* right-hand sides per block solve; more transmitters are solved in
                             blocks of this width (Krylov memory grows with it) [64] */
    int32_t sweep_engine; /* MIXED modes, engine of the complex FP32 ORAS sweeps:
                             0 = default (4); 1 = tensor cores (mma.sync), operands split into
                             two TF32 parts (about FP32 accuracy); 2 = tensor cores (mma.sync),
                             plain TF32; 3 = CUDA cores, FP32; 4 = fifth-generation tensor
                             cores (tcgen05, TF32 operands, accumulators in tensor memory) fed
                             by bulk copies from two tiled copies of the factor panels (about
                             2.4 GB per GB of panels more device memory).  TF32 engines carry
                             ~1e-3 relative rounding in the preconditioner, absorbed by the
                             outer FGMRES */
    int32_t block_krylov; /* 0 = pseudo-block FGMRES: every column of a block keeps its own
                             Krylov space and the columns' operations are fused (Section 6.3)
                             [0]; 1 = true block FGMRES (the block methods of Section 7): one
                             Krylov space shared by the columns of a block, built by block
                             Arnoldi with block classical Gram-Schmidt (twice) and Cholesky QR
                             (twice), complex FP64 vectors, blocks of at most 32 columns (a
                             column whose new direction falls below 1e-7 of its norm is
                             deflated); the preconditioner is the ORAS of `precision`.
                             iters_max then counts block steps.  Other values: MWI_EINVAL */
    int32_t recycle;      /* 1 = Krylov recycling across a sequence of nearby systems (the
                             recycling of Section 7): a forward solve whose transmitter count
                             m <= 32 equals the previous converged forward solve's starts every
                             column from the least-residual element of the span of the previous
                             forward solutions (FP32 projection, x0 = X Y,
                             Y = argmin ||B - A X Y||); an adjoint solve uses the span of the
                             current forward solutions and, when the previous adjoint solve had
                             the same m, of the previous adjoint solutions (when the receivers
                             are among the transmitters the adjoint solution lies in the first
                             span).  The solve then runs to rtol as usual, and iters_max is 0
                             when the guess already meets it.  Its SpMM counts in the SpMM timer and
                             its projection in the orthogonalisation timer.  0 = off [0];
                             other values: MWI_EINVAL */
    int32_t factor_reuse; /* mwi_update_eps[_device]: up to this many consecutive updates
                             reassemble A for the new eps_r but keep the previous subdomain
                             factors as the ORAS preconditioner (a preconditioner for a
                             nearby operator: more iterations, same rtol on the new system);
                             the next update refactors.  0 = refactor on every update [0];
                             < 0: MWI_EINVAL */
} mwi_solver_opts;

typedef struct {
    int32_t iters_max;    /* largest outer iteration count over columns */
    int32_t inner_total;  /* MIXED_NESTED: inner iterations summed over outer steps */
    int32_t n_converged;  /* columns whose true relative residual <= rtol */
    int32_t n_perturbed;  /* pivots perturbed in the factorisation */
    double resid_max;     /* largest true relative residual over columns */
    double setup_ms;      /* assemble + factorise (mwi_assemble only) */
    double solve_ms;      /* FGMRES wall time of this call */
} mwi_solve_info;

/* ---------------------------------------------------------------------- */
/* Mesh: Section 2.1 (edge elements on a tetrahedral mesh).
 * xyz [nv*3] vertex coordinates (m); tet [nt*4] vertex ids; bface_tag [nt*4]
 * tag of the face opposite local vertex k: 0 interior, 1 perfectly conducting
 * (Eq. eqmetal: its DOFs are removed), 2 impedance (Eq. eqwgi with
 * beta = k0 sqrt(eps_r) of the owning tet).  order = 1 (Whitney, 6 DOFs/tet)
 * or 2 (hierarchical first kind, 20 DOFs/tet).  Builds edges/faces, DOF
 * numbering, and the element geometric integrals on the current device.
 * Returns MWI_EINVAL for a degenerate tet or bad ids. */
mwi_status mwi_mesh_create(const double* xyz, int64_t nv, const int32_t* tet, int64_t nt,
                           const int32_t* bface_tag, int32_t order, mwi_mesh_t* out);

/* Number of DOFs after PEC removal. */
mwi_status mwi_mesh_ndof(mwi_mesh_t mesh, int64_t* ndof);

/* Identity of every DOF in the library's internal order: kind[ndof]
 * (0 Whitney edge, 1 edge gradient, 2 face lambda_c N_ab, 3 face lambda_a N_bc)
 * and verts[ndof*3] (global vertex ids in increasing order; third = -1 for
 * edge DOFs).  Lets a caller map fields to its own numbering. */
mwi_status mwi_mesh_dof_keys(mwi_mesh_t mesh, int32_t* kind, int64_t* verts);

/* Destroys a mesh; MWI_ESTATE if a problem still references it. */
mwi_status mwi_mesh_destroy(mwi_mesh_t mesh);

/* ---------------------------------------------------------------------- */
/* Assemble A = K - k0^2 sum_t eps_t M_t + i sum_f beta_f B_f (Eq. pbdirectvarf,
 * Eq. linsys) for eps_r [nt] (interleaved complex, host) at freq_hz, build the
 * ORAS decomposition of Section 3 (partition, delta-overlap, P1 partition of
 * unity interpolated at edge midpoints, local operators B_i with impedance
 * transmission conditions, k = k0 sqrt(eps_t) of the owning tet) and factorise
 * every B_i as one batch (LDL^T, nested-dissection multifrontal, FP64 or
 * FP32 per opts.precision).  cuda_stream: a cudaStream_t (0 = default). */
mwi_status mwi_assemble(mwi_mesh_t mesh, const double* eps_r, double freq_hz,
                        const mwi_solver_opts* opts, void* cuda_stream, mwi_problem_t* out);

/* Same as mwi_assemble but eps_r [nt] (interleaved complex) is a device array. */
mwi_status mwi_assemble_device(mwi_mesh_t mesh, const double* eps_r_dev, double freq_hz,
                               const mwi_solver_opts* opts, void* cuda_stream, mwi_problem_t* out);

/* Re-assemble and re-factorise an existing problem for new eps_r (host) at the
 * same frequency and options, reusing its decomposition and workspaces. */
mwi_status mwi_update_eps(mwi_problem_t prob, const double* eps_r);
mwi_status mwi_update_eps_device(mwi_problem_t prob, const double* eps_r_dev);

/* ---------------------------------------------------------------------- */
/* Forward problems (Eq. linsys, one column per transmitter) solved together
 * by pseudo-block FGMRES + ORAS, then S_ij = conj(q_i^T u_j) / |q_i|^2 with
 * q_i = s_i e_{k_i} (Eq. sij for edge-current receivers).  S_out
 * [n_rx*n_tx] interleaved complex, column-major (S_out[i + n_rx*j]).  The
 * fields stay resident for mwi_misfit_and_gradient and mwi_fields_device.
 * info may be NULL. */
mwi_status mwi_forward_solve(mwi_problem_t prob, const mwi_antenna* tx, int32_t n_tx,
                             const mwi_antenna* rx, int32_t n_rx, double* S_out,
                             mwi_solve_info* info);

/* Misfit J = 1/2 sum_ij w_ij |S_ij - S_meas_ij|^2 (Eq. defJ; w = 1 when w is
 * NULL, Eq. defJ2's normalisation when w_ij = 1/|S_empty_ij|^2) for the S of
 * the last mwi_forward_solve, the adjoint solve of Eq. pbadj with the same
 * factors, and dJ_deps [nt] interleaved = dJ/dRe(eps_t) + i dJ/dIm(eps_t)
 * (Section 5; includes the boundary term from beta = k0 sqrt(eps_t) on
 * impedance faces).  S_meas, w: [n_rx*n_tx] column-major, host.
 * MWI_ESTATE without a prior forward solve. */
mwi_status mwi_misfit_and_gradient(mwi_problem_t prob, const double* S_meas, const double* w,
                                   double* J_out, double* dJ_deps, mwi_solve_info* info);

/* Misfit only: J (Eq. defJ) for the S of the last forward solve, no adjoint
 * solve.  S_meas, w host arrays as above. */
mwi_status mwi_misfit(mwi_problem_t prob, const double* S_meas, const double* w, double* J_out);

/* Same with device arrays: S_meas_dev, w_dev (nullable), dJ_deps_dev; J_out host. */
mwi_status mwi_misfit_and_gradient_device(mwi_problem_t prob, const double* S_meas_dev,
                                          const double* w_dev, double* J_out,
                                          double* dJ_deps_dev, mwi_solve_info* info);

/* Borrowed device view of the last fields U [n][m] (row-major: m = n_tx
 * contiguous complex values per DOF, internal DOF order of mwi_mesh_dof_keys).
 * which = 0 forward fields, 1 adjoint fields.  Valid until the next call on
 * the handle. */
mwi_status mwi_fields_device(mwi_problem_t prob, int32_t which, void** dev_ptr, int64_t* n,
                             int64_t* m);

/* Copy the last fields (as mwi_fields_device describes them) to the host
 * array out [n*m*2] (interleaved complex, row-major [n][m]). */
mwi_status mwi_copy_fields(mwi_problem_t prob, int32_t which, double* out);

mwi_status mwi_problem_destroy(mwi_problem_t prob);

/* Thread-local message for the last non-OK status of this thread. */
const char* mwi_last_error(void);

/* ---------------------------------------------------------------------- */
/* Building blocks exposed for testing and measurement.  All vectors are
 * device arrays of complex double, row-major [n][m] (m contiguous). */

/* y = A x for the assembled global matrix (the complex SpMM of every FGMRES
 * iteration). */
mwi_status mwi_spmm_device(mwi_problem_t prob, const double* x_dev, double* y_dev, int32_t m);

/* y = M^-1 x with the problem's preconditioner in its precision (x and y in
 * FP64; converted around the FP32 factors if MIXED): the ORAS of Eq. ORAS, or
 * the two-level ORAS once mwi_set_coarse_space has given the problem a
 * coarse space. */
mwi_status mwi_oras_apply_device(mwi_problem_t prob, const double* x_dev, double* y_dev,
                                 int32_t m);

/* Allocation-free variant of mwi_oras_apply_device, for callers that cannot
 * call cudaMalloc while they run: processes whose device memory is all handed
 * to a pool allocator (for example PyTorch's caching allocator in a serving
 * process that reserves the GPU up front), or latency-critical loops that must
 * not pay cudaMalloc's implicit device synchronisation.  The paper has no
 * counterpart; this is a deployment aid.
 * Same arguments and result as mwi_oras_apply_device.  Its scratch (local
 * vectors, update vectors, FP32 copies in the MIXED path) lives in one
 * file-scope device array of 32 MiB that every GPU loading the library holds
 * until the process exits; the call allocates nothing (no cudaMalloc, no
 * cudaFree, no allocating library routine).  A problem whose scratch need
 * exceeds 32 MiB -- (2 * n_local + n_update_rows) * m complex values in the
 * factor precision, plus 2 * n * m FP32 complex values when MIXED -- is
 * rejected with MWI_EINVAL before any launch.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, once per device); make that first call before any
 * stream capture.  All calls share the array: calls that overlap on the GPU
 * (different streams, threads or processes' contexts on one device) race and
 * must be serialised by the caller. */
mwi_status mwi_oras_apply_device_noalloc(mwi_problem_t prob, const double* x_dev, double* y_dev,
                                         int32_t m);

/* Global CSR of A: row_ptr [n+1] (host), col [nnz] (host), val [2*nnz] (host). */
mwi_status mwi_matrix_csr(mwi_problem_t prob, int64_t* nnz, int64_t* row_ptr, int32_t* col,
                          double* val);

/* Decomposition summary: part [nt] (host), and per subdomain the number of
 * local DOFs n_local [n_sub] (host).  Either pointer may be NULL. */
mwi_status mwi_decomposition(mwi_problem_t prob, int32_t* part, int64_t* n_local);

/* Factor statistics: total factor entries, front count, largest front. */
mwi_status mwi_factor_stats(mwi_problem_t prob, int64_t* factor_entries, int64_t* n_fronts,
                            int64_t* max_front, double* factor_flops);

/* Nodal (P1) permittivity parameter (Section 6.3: a piecewise-linear parameter
 * on the state mesh).  kappa_dev [nv] (device, interleaved complex, the
 * caller's vertex numbering) holds a relative permittivity per vertex; the
 * field kappa(x) = sum_v kappa_v lambda_v(x) varies inside every tet, so the
 * mass term of Eq. pbdirectvarf becomes
 *     int_t kappa N_i . N_j = sum_w kappa_{v_w} int_t lambda_w N_i . N_j
 * (four vertex-weighted element masses per tet, closed forms, built on the
 * mesh's first use of this call and kept with the mesh).  beta on impedance
 * faces and the interface wavenumber of the ORAS local problems take the P1
 * field at the owning tet's centroid, 1/4 sum of its vertex values (the paper
 * does not say; this is the library's reading).  Reassembles A and, as
 * mwi_update_eps does (including opts.factor_reuse), the subdomain factors.
 * Until the next mwi_update_eps[_device] the problem is in nodal-parameter
 * mode: mwi_misfit_and_gradient[_device] return MWI_ESTATE and
 * mwi_misfit_and_gradient_kappa_device gives the gradient.  Errors:
 * MWI_EINVAL for a null pointer or a non-finite kappa (checked on the device
 * before anything changes). */
mwi_status mwi_update_kappa_device(mwi_problem_t prob, const double* kappa_dev);

/* Objective of Eq. defJ2 for the nodal parameter: J = 1/2 sum_ij w_ij
 * |S_ij - S_meas_ij|^2 (w_dev nullable: w = 1; the normalised misfit takes
 * w_ij = 1/|S_empty_ij|^2, see mwi_normalised_weights) for the S of the last
 * forward solve, and the penalty R = (alpha/2) int |grad kappa|^2 =
 * (alpha/2) Re(kappa^H K kappa) (K the P1 stiffness matrix).  Runs the adjoint
 * solve (Eq. pbadj) with the same factors and writes to dPhi_dkappa_dev [nv]
 * (device, interleaved) the gradient of J + R with respect to the vertex
 * values, dPhi/dRe kappa_v + i dPhi/dIm kappa_v: per (tet, vertex) the term
 * k0^2 sum_j lambda_j^T M_t^(w) u_j plus a quarter of the tet's beta term,
 * conjugated and summed over the vertex's tets (ascending), plus
 * alpha (K kappa)_v.  J_out and R_out (nullable) are host scalars; S_meas_dev
 * and w_dev are [n_rx*n_tx] column-major device arrays.  MWI_ESTATE without
 * a prior mwi_update_kappa_device and forward solve; MWI_EINVAL for alpha < 0;
 * MWI_ENOTCONV still fills every output. */
mwi_status mwi_misfit_and_gradient_kappa_device(mwi_problem_t prob, const double* S_meas_dev,
                                                const double* w_dev, double alpha, double* J_out,
                                                double* R_out, double* dPhi_dkappa_dev,
                                                mwi_solve_info* info);

/* Weights of the normalised misfit of Eq. defJ2: w[e] = 1 / |S_empty[e]|^2
 * for count complex entries (host arrays; S_empty interleaved, as
 * mwi_forward_solve returns it for the empty -- gel-filled -- chamber).
 * MWI_EINVAL if an entry is zero or not finite. */
mwi_status mwi_normalised_weights(const double* S_empty, int64_t count, double* w_out);

/* Algorithmic memory traffic of one ORAS application (Eq. ORAS) to m columns,
 * in bytes, for the roofline of the sweeps (no counterpart in the paper; a
 * measurement aid): every stored factor entry read once per sweep (the unit
 * lower triangles of L11^-1 and the blocks -L21 L11^-1) plus D^-1, and the
 * vectors each step must move -- the gather of x into the local vectors, per
 * front the pivot rows read and written in both sweeps, the update rows
 * written once and read by the parent (forward) and the ancestor rows read
 * (backward), and the weighted scatter into y.  Entries count 8 bytes in the
 * complex FP32 modes and 16 in FP64. */
mwi_status mwi_oras_traffic(mwi_problem_t prob, int32_t m, double* bytes);

/* Device memory held by a problem: its operator, subdomain factors, field
 * blocks and solver workspaces (buffers grow with the widest solve so far);
 * the mesh and its decomposition, shared by the problems on that mesh, are not
 * counted.  For admission against a memory budget (a serving cache). */
mwi_status mwi_problem_device_bytes(mwi_problem_t prob, int64_t* bytes);

/* Per tree level of the multifrontal sweeps (deepest level first; a
 * measurement aid, no counterpart in the paper): *n_levels levels; for the
 * first max_levels of them the fronts, the partitioned-inverse panel entries
 * (sum f p), the update rows (sum u), and the 128-row tiles of the forward
 * (rows) and backward (pivots) tensor-core products.  Array arguments may be
 * NULL. */
mwi_status mwi_sweep_levels(mwi_problem_t prob, int32_t max_levels, int32_t* n_levels, int64_t* fronts,
                            int64_t* panel_entries, int64_t* update_rows, int64_t* tiles_fwd,
                            int64_t* tiles_bwd);

/* Krylov recycling across problems (the recycling of Section 7, across the
 * nearby frequencies of a multi-frequency measurement or of a serving cache):
 * the resident forward solutions of src (and its adjoint solutions, if any)
 * become the recycled space of dst, so that dst's next forward solve with the
 * same transmitter count (at most 32) starts every column from the
 * least-residual element of their span, and its next adjoint solve from the
 * span of its own forward solutions and of src's adjoint solutions, exactly as
 * after a solve of dst itself (see recycle in mwi_solver_opts).  Both problems
 * must be on the same mesh; dst must have recycle = 1 (else MWI_ESTATE); src
 * must hold forward solutions (else MWI_ESTATE).  Copies on dst's stream and
 * returns when done; dst's previous fields are dropped.  The two handles must
 * not be in use by other threads during the call. */
mwi_status mwi_recycle_from(mwi_problem_t dst, mwi_problem_t src);

/* Two-level ORAS (Section 7: a coarse space keeps the iteration count of the
 * one-level method from growing with the number of subdomains).  The coarse
 * space is the lowest-order Whitney space of coarse_mesh (order 1, covering
 * the same domain; its PEC faces remove coarse DOFs as in any mesh).
 * Prolongation P [n x n_c], real: the fine edge e's tangential integral of a
 * coarse field by the midpoint rule, P[e,E] = N_E(m_e) . (x_hi - x_lo), with
 * N_E evaluated in the lowest-numbered coarse tet that holds the midpoint m_e
 * (smallest barycentric coordinate >= -1e-12); for a midpoint outside the
 * coarse mesh, in the lowest-numbered tet whose smallest barycentric
 * coordinate is within 1e-12 of the largest over all tets (the affine
 * extension of the least-outside tet's basis); only the fine Whitney DOFs get
 * rows. 
 * Coarse operator A_c = P^T A P (Galerkin; A complex symmetric), factorised as
 * one dense front in the problem's factor precision.  Preconditioner (every
 * solve of the problem, and mwi_oras_apply_device):
 *   M_2 r = M_ORAS (r - A Q r) + Q r,   Q = P A_c^{-1} P^T.
 * A_c and its factors follow every later refactorisation (new eps_r, kappa).
 * Setup: P and the pattern of A_c on the host cores, A_c's values from a host
 * copy of A (host cores), the factorisation on the problem's stream; returns
 * when done.  n_c <= 16384 (else MWI_EINVAL; the dense front takes n_c^2
 * complex entries twice).  coarse_mesh may be destroyed afterwards.  NULL
 * removes the coarse space.  mwi_oras_apply_device_noalloc refuses a problem
 * with a coarse space (MWI_EINVAL). */
mwi_status mwi_set_coarse_space(mwi_problem_t prob, mwi_mesh_t coarse_mesh);

/* Host-only form of the prolongation of mwi_set_coarse_space (no device
 * work), for checking the host logic without a GPU: the fine mesh (order 1 or
 * 2) and the coarse mesh (order 1) as mwi_mesh_create takes them; *n, *nc, *nnz
 * the fine and coarse DOF counts and the entries of P; P in CSR (p_rp [n+1],
 * p_col [nnz], p_val [nnz]) in the library's DOF numbering of each mesh, with
 * the DOF keys of both numberings as mwi_mesh_dof_keys gives them (fkind [n],
 * fverts [3n], ckind [nc], cverts [3nc]).  Call with null arrays to get the
 * sizes; every array may be NULL. */
mwi_status mwi_coarse_prolongation_host(const double* fxyz, int64_t fnv, const int32_t* ftet, int64_t fnt,
                                        const int32_t* fbface_tag, int32_t forder, const double* cxyz, int64_t cnv,
                                        const int32_t* ctet, int64_t cnt, const int32_t* cbface_tag, int64_t* n,
                                        int64_t* nc, int64_t* nnz, int64_t* p_rp, int32_t* p_col, double* p_val,
                                        int32_t* fkind, int64_t* fverts, int32_t* ckind, int64_t* cverts);

/* Host-only form of the antenna map of mwi_forward_solve (no device work),
 * for checking it without a GPU: the mesh as mwi_mesh_create takes it; for
 * every antenna (the mwi_antenna rule) the DOF id of its edge in the library's
 * DOF numbering (dof_out [n_ant]) and its sign (sign_out [n_ant]: +1 when dir
 * agrees with the edge's orientation from the lower to the higher vertex id,
 * else -1); *ndof and the DOF keys (kind [ndof], verts [3 ndof]) as
 * mwi_mesh_dof_keys gives them.  MWI_EINVAL for an antenna whose edge is a
 * removed PEC edge, a zero or non-finite dir or a non-finite pos.  Call with
 * null arrays to get *ndof; every array may be NULL. */
mwi_status mwi_antenna_map_host(const double* xyz, int64_t nv, const int32_t* tet, int64_t nt,
                                const int32_t* bface_tag, int32_t order, const mwi_antenna* ants, int32_t n_ant,
                                int32_t* dof_out, double* sign_out, int64_t* ndof, int32_t* kind, int64_t* verts);

/* Host-only form of the decomposition of Section 3 (no device work), for
 * checking its host logic without a GPU: the mesh as mwi_mesh_create takes
 * it, and n_sub, overlap and nd_leaf as in mwi_solver_opts (0: the defaults).
 * Out (every pointer may be NULL; call with null arrays to get the sizes):
 * part [nt] the non-overlapping partition; sub_off [n_sub+1] offsets of each
 * subdomain's local rows in loc2glob [nloc] (global DOF ids, the subdomain's
 * nested-dissection order) and dweight [nloc] (the partition-of-unity weight
 * D_i of each local row, Eq. algebPartUnity); fu_off [n_sub+1] offsets of each
 * subdomain's boundary face uses (the faces of T_i^delta with no neighbour in
 * T_i^delta that are not PEC: the outer impedance faces and the interface
 * faces that carry the impedance condition of B_i) in fu_verts [3 nfu] (the
 * face's sorted vertex ids) and fu_tet [nfu] (the tet of T_i^delta owning it);
 * *nloc, *nfu, *ndof and the DOF keys (kind [ndof], verts [3 ndof]) as
 * mwi_mesh_dof_keys gives them; *factor_entries and *upd_rows, the
 * multifrontal factor's entries (sum f p) and update rows (sum u). */
mwi_status mwi_decomposition_host(const double* xyz, int64_t nv, const int32_t* tet, int64_t nt,
                                  const int32_t* bface_tag, int32_t order, int32_t n_sub, int32_t overlap,
                                  int32_t nd_leaf, int32_t* part, int64_t* sub_off, int32_t* loc2glob,
                                  double* dweight, int64_t* fu_off, int32_t* fu_verts, int32_t* fu_tet,
                                  int64_t* nloc, int64_t* nfu, int64_t* ndof, int32_t* kind, int64_t* verts,
                                  int64_t* factor_entries, int64_t* upd_rows);

/* Host-only form of the multifrontal structure of the decomposition (the
 * same arguments as mwi_decomposition_host): *n_fronts fronts over all
 * subdomains, children before parents, with front_info [5 n_fronts] = (sub,
 * start, p, u, parent) per front (start: first pivot, local nested-dissection
 * index; p pivots; u update rows; parent: front id or -1), u_off [n_fronts]
 * offsets of each front's update-row list in urows [*n_urows] (local
 * nested-dissection indices of ancestor pivots, ascending) and urel
 * [*n_urows] (each update row's position among its parent's front rows:
 * pivots, then update rows).  The extend-add table of the sweeps: for front
 * row t of front s (index sum over the fronts before s of p + u, plus t),
 * asm_ptr [sum (p+u) + 1] delimits in asm_src [*n_asm] the rows of the update
 * buffer (front c's update row j is row sum over the fronts before c of u,
 * plus j) that add into it, children ascending.  Every pointer may be NULL;
 * call with null arrays to get the sizes. */
mwi_status mwi_fronts_host(const double* xyz, int64_t nv, const int32_t* tet, int64_t nt, const int32_t* bface_tag,
                           int32_t order, int32_t n_sub, int32_t overlap, int32_t nd_leaf, int32_t* n_fronts,
                           int64_t* n_urows, int64_t* n_asm, int32_t* front_info, int64_t* u_off, int32_t* urows,
                           int32_t* urel, int64_t* asm_ptr, int32_t* asm_src);

/* Host-only form of the assembly map of A (no device work): the pattern of A
 * in CSR (row_ptr [ndof+1], col [nnz]) in the library's DOF numbering and, per
 * stored entry, its element contributions in summation order (slot_ptr
 * [nnz+1], contrib [ncontrib]: bits 0..15 the packed local pair (i <= j:
 * i nl - i (i-1)/2 + j - i), bits 16..61 the tet id or face-use id, bit 62
 * set for a face use); the local DOFs of every tet (tet_dofs [nt nl], -1 for
 * a removed PEC DOF, nl = 6 or 20) and of every face use (fu_dofs [nfu nlf],
 * nlf = 3 or 8) with its owning tet (fu_tet [nfu]) and sorted vertex ids
 * (fu_verts [3 nfu]); *ndof and the DOF keys (kind [ndof], verts [3 ndof]).
 * The device assembly sums exactly these contributions in this order.  Every
 * pointer may be NULL; call with null arrays to get the sizes. */
mwi_status mwi_slots_host(const double* xyz, int64_t nv, const int32_t* tet, int64_t nt, const int32_t* bface_tag,
                          int32_t order, int64_t* ndof, int64_t* nnz, int64_t* ncontrib, int64_t* nfu,
                          int64_t* row_ptr, int32_t* col, int64_t* slot_ptr, int64_t* contrib, int32_t* tet_dofs,
                          int32_t* fu_dofs, int32_t* fu_tet, int32_t* fu_verts, int32_t* kind, int64_t* verts);

/* Host-only form of the local operators' assembly maps (the same mesh and
 * decomposition arguments as mwi_decomposition_host): the block-diagonal
 * pattern of the B_i (B_row_ptr [nloc+1] over the concatenated local rows of
 * mwi_decomposition_host's loc2glob, B_col [nslot] the column's local
 * nested-dissection index within its subdomain), each stored entry's
 * contributions in summation order (B_slot_ptr [nslot+1], B_contrib
 * [ncontrib], encoded as in mwi_slots_host, face-use ids indexing the face
 * uses of mwi_decomposition_host) and the face uses' face-local DOFs (fu_dofs
 * [nfu nlf]); and the map that assembles the fronts from them
 * (amap_front_ptr [n_fronts+1] over the fronts of mwi_fronts_host,
 * amap_slot [namap] the stored entry, amap_pos [namap] its position in the
 * factor store: the front's panel offset (sum of (p+u) p over the fronts
 * before it) + pivot column * (p+u) + front row).  Every pointer may be NULL;
 * call with null arrays to get the sizes. */
mwi_status mwi_local_assembly_host(const double* xyz, int64_t nv, const int32_t* tet, int64_t nt,
                                   const int32_t* bface_tag, int32_t order, int32_t n_sub, int32_t overlap,
                                   int32_t nd_leaf, int64_t* nloc, int64_t* nslot, int64_t* ncontrib, int64_t* nfu,
                                   int64_t* namap, int32_t* n_fronts, int64_t* B_row_ptr, int32_t* B_col,
                                   int64_t* B_slot_ptr, int64_t* B_contrib, int32_t* fu_dofs,
                                   int64_t* amap_front_ptr, int64_t* amap_slot, int64_t* amap_pos);

/* Sizes of the problem's coarse space (all 0 without one): n_c coarse DOFs,
 * entries of P and of A_c, host+device setup time of the last (re)build of
 * A_c and its factors, and the factorisation's replaced pivots.  Any pointer
 * may be NULL. */
mwi_status mwi_coarse_info(mwi_problem_t prob, int64_t* n_coarse, int64_t* nnz_p, int64_t* nnz_ac,
                           double* setup_ms, int32_t* n_perturbed);

/* Host copies of P (CSR: p_rp [n+1], p_col [nnz_p], p_val [nnz_p]) and of A_c
 * (CSR: ac_rp [n_c+1], ac_col [nnz_ac], ac_val [2*nnz_ac] interleaved complex),
 * columns ascending in every row.  Any pointer may be NULL; MWI_ESTATE
 * without a coarse space. */
mwi_status mwi_coarse_operator(mwi_problem_t prob, int64_t* p_rp, int32_t* p_col, double* p_val, int64_t* ac_rp,
                               int32_t* ac_col, double* ac_val);

/* Upper estimate of the device bytes a problem on this mesh with these
 * options will hold after solves of n_rhs transmitters (its operator,
 * factors, field blocks and solver workspaces, as mwi_problem_device_bytes
 * counts them), computed on the host before the problem exists: builds (or
 * reuses) the mesh's decomposition and symbolic factorisation, which the
 * problem would build anyway, and allocates only the mesh's shared operator
 * structure.  For admission against a memory budget before building a
 * problem on a mesh not seen yet (no counterpart in the paper). */
mwi_status mwi_problem_estimate_bytes(mwi_mesh_t mesh, const mwi_solver_opts* opts, int32_t n_rhs,
                                      int64_t* bytes);

/* Per-kernel timing since the last reset, from CUDA events recorded on the
 * problem's stream around every call (no synchronisation in between):
 * ms[0] SpMM, ms[1] ORAS apply, ms[2] orthogonalisation (CGS2 + norms),
 * ms[3] factorisation; counts[4] calls of each.  Enabled by opts.verbose >= 2.
 * reset != 0 clears the accumulators after reading. */
mwi_status mwi_kernel_times(mwi_problem_t prob, double* ms, int64_t* counts, int32_t reset);

/* Number of kernels this library has launched in the process so far. */
int64_t mwi_launch_count(void);

/* Number of device allocations (cudaMalloc calls) this library has made in
 * the process so far, successful or not; lets a caller check that a call
 * allocated nothing. */
int64_t mwi_device_alloc_count(void);

#ifdef __cplusplus
}
#endif

#endif /* MWI_H */
