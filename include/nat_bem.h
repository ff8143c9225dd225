/*
 * nat_bem.h -- C ABI of the GB300 (sm_103a) exterior Helmholtz Burton-Miller BEM solver.
 *
 * The problem (paper Sec. 3.4): given a closed triangle mesh, a wavenumber k and Neumann data
 * (normal derivative of the pressure, constant per triangle), solve for the surface Dirichlet
 * data (pressure) and then evaluate the radiated pressure at field points. The boundary
 * integral equation is the Burton-Miller combination of Sec. 4, Eq. 6, with the free-space
 * Green's function G(x,y) = e^{ikr}/(4 pi r) of Sec. 4.2 and coupling beta = i/k. It is
 * discretised with piecewise-constant elements collocated at the centroids:
 *
 *   L p = R g,   L_ij = 1/2 d_ij - int_j [dG/dn_y + beta d2G/dn_x dn_y] dS_y,
 *                R_ij = -int_j [G + beta dG/dn_x] dS_y - (beta/2) d_ij,
 *
 * which is the directly assembled two-matrix system "A g = B p" of Sec. 4.1. The linear solve
 * is GMRES stopped at a relative residual of 1e-6 within 200 iterations (the paper's solver
 * settings, Sec. 6.1). The field follows from the exterior representation
 * p(x) = int [p dG/dn_y - G g] dS_y (Sec. 3.4: pressure anywhere from the Neumann and
 * Dirichlet data).
 *
 * Conventions for every call:
 *   - Triangles wind counter-clockwise seen from outside (outward normals).
 *   - Complex arrays are single-precision complex (float re, float im) interleaved. A block of
 *     nrhs right-hand sides is column-major: column s holds nt (or m) consecutive values.
 *   - Array arguments may be host or device pointers; the library detects which. With host
 *     pointers the call copies through the given stream and returns once the copy is done.
 *   - `cuda_stream` is a cudaStream_t (NULL = the legacy default stream). All device work of
 *     a call is ordered on it.
 *   - The caller owns every array it passes. The library owns nat_bem_op (the device-resident
 *     operator, geometry and Krylov workspace) until nat_bem_destroy.
 *   - Calls on one op are not thread-safe; different ops are independent.
 *   - No function throws or aborts across the ABI. On any status other than NAT_BEM_OK,
 *     nat_bem_last_error() returns a message (thread-local) and outputs are untouched, except
 *     NAT_BEM_ENOCONV, which still writes the best iterate and fills the info struct.
 */
#ifndef NAT_BEM_H
#define NAT_BEM_H

#include <stdint.h>

#if defined(__GNUC__)
#define NAT_BEM_API __attribute__((visibility("default")))
#else
#define NAT_BEM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NAT_BEM_OK = 0,
  NAT_BEM_EINVAL = 1,   /* bad argument or invalid mesh (see nat_bem_assemble)            */
  NAT_BEM_ENOMEM = 2,   /* device allocation failed or the op would exceed a memory budget */
  NAT_BEM_ENOCONV = 3,  /* GMRES did not reach tol within max_iter (best iterate returned)  */
  NAT_BEM_ECUDA = 4,    /* a CUDA call failed; the message holds the CUDA error string      */
  NAT_BEM_ETIMEOUT = 5, /* a bounded wait gave up                                           */
  NAT_BEM_EBUSY = 6     /* the resource is in use (serving)                                 */
} nat_bem_status;

typedef enum {
  NAT_BEM_PREC_FP32 = 0,       /* FP32 operator and matvec, FP64 Gram-Schmidt / least squares */
  NAT_BEM_PREC_MIXED_TF32 = 1, /* inner GMRES products in TF32, FP64-refined FP32 residual    */
  NAT_BEM_PREC_MIXED_BF16 = 2, /* inner GMRES on a BF16 operator copy, FP64-refined residual   */
  NAT_BEM_PREC_MIXED_FP16 = 3  /* inner GMRES on an FP16 operator copy, each row scaled by a     */
                               /* power of two into FP16's range (the same bytes as BF16, 3 more */
                               /* significant bits, so refinement sweeps contract further)      */
} nat_bem_precision;

/*
 * Solver and quadrature options (paper Sec. 6.1 gives the solver settings: tolerance 1e-6, at
 * most 200 iterations; Sec. 4.1 says only "Gaussian quadrature", so the rules are this
 * library's choice, stated here).
 */
typedef struct {
  int32_t adj_subdiv_levels; /* vertex-sharing pairs: 7-point rule on 4^levels sub-triangles (2) */
  int32_t self_theta_pts;    /* self pair: Gauss-Legendre points per edge in the angle (16)      */
  double tol;                /* relative residual ||b - L p|| / ||b|| to stop at (1e-6)         */
  int32_t max_iter;          /* GMRES iterations (plain), total inner iterations (mixed) (200); */
                             /* at most 255 unrestarted, 100000 with restart > 0                */
  nat_bem_precision prec;    /* arithmetic of the solve (NAT_BEM_PREC_FP32)                      */
  int32_t inner_max_iter;    /* mixed: iterations per inner solve (60)                            */
  double inner_tol;          /* mixed: relative tolerance of each inner solve (1e-2). A sweep    */
                             /* near the end asks only for the contraction still missing,        */
                             /* 0.7 tol / (largest open relative residual), where that is looser: */
                             /* inner_tol x 2^e for the largest e <= 5 that stays within it       */
  int32_t max_refinements;   /* mixed: outer refinement sweeps (10)                               */
  int32_t restart;           /* GMRES(m): Krylov vectors kept, m in 1..255; 0 = unrestarted (0).  */
                             /* The basis takes 16 nt nrhs (m + 1) bytes instead of             */
                             /* 16 nt nrhs (max_iter + 1): the lever for serving memory          */
  int32_t quad_regular;      /* points of the rule on pairs sharing no vertex: 7 (Radon's degree- */
                             /* 5 rule) is the only value (7)                                      */
  int32_t device_loop;       /* 1: each GMRES run goes to convergence on the device (a CUDA graph */
                             /* whose conditional loop repeats captured iterations), so a plain  */
                             /* solve makes one host sync; 0: chunks of iterations with a host    */
                             /* check after each (1). The batch driver and the server use 0 when  */
                             /* they run several workers (other streams fill those gaps)          */
} nat_bem_opts;

typedef struct nat_bem_op nat_bem_op; /* opaque */

typedef struct {
  int32_t iterations;   /* GMRES iterations (mixed: summed over inner solves), max over RHS   */
  int32_t refinements;  /* mixed: outer sweeps done; restarted: GMRES cycles; else 0            */
  double rel_residual;  /* largest ||b - L p|| / ||b|| over the RHS (FP64 accumulation)        */
} nat_bem_solve_info;

/* Fills *opts with the defaults listed above. */
NAT_BEM_API void nat_bem_opts_default(nat_bem_opts* opts);

/*
 * Assembles L and R (Sec. 4, Eq. 6; Sec. 4.1) for mesh (verts, tris) at wavenumber k.
 *   verts: nv x 3 float64, row-major.  tris: nt x 3 int32 vertex indices, row-major.
 *   k: wavenumber (> 0, finite).  opts: NULL for defaults.  *out: receives the new op.
 * Work: geometry on the device, FP32 regular element pairs, FP64 self and vertex-sharing
 * pairs. The op keeps L and R (8 nt^2 bytes each, complex64, leading dimension nt rounded up
 * to 32) plus a BF16 copy of L for NAT_BEM_PREC_MIXED_BF16 (4 nt^2 bytes), or an FP16 copy with
 * one power-of-two scale per row for NAT_BEM_PREC_MIXED_FP16 (4 nt^2 + 4 nt bytes). Returns when the
 * work is enqueued (the mesh checks run on the host before).
 * NAT_BEM_EINVAL: nv or nt <= 0, an index out of range, a non-finite coordinate, a zero-area
 * triangle, a mesh that is not closed with every edge used once in each direction, negative
 * enclosed volume (inward winding), k <= 0 or not finite, opts out of range.
 * NAT_BEM_ENOMEM: the device allocations failed.
 */
NAT_BEM_API nat_bem_status nat_bem_assemble(const double* verts, int64_t nv, const int32_t* tris, int64_t nt,
                                double k, const nat_bem_opts* opts, void* cuda_stream,
                                nat_bem_op** out);

/*
 * Galerkin form (paper Sec. 4, Eq. 6 tested with the P1 hat functions; the element-to-element
 * integration of Sec. 4.1, as bempp does it): P1 (continuous, piecewise linear) Dirichlet data
 * p at the nv vertices, P0 Neumann data g per triangle, P1 test functions psi_i:
 *
 *   L p = R g,   L = 1/2 M11 - K - beta H  (nv x nv),   R = -V - beta K' - (beta/2) M10  (nv x nt),
 *   H_ij = int int G(x, y) [k^2 (n_x . n_y) phi_j(y) psi_i(x) - curl phi_j(y) . curl psi_i(x)],
 *
 * the hypersingular term in Maue's integrated-by-parts form (curl u = n x grad u, constant per
 * triangle for P1), M11 and M10 the P1-P1 and P0-P1 mass matrices, K, K', V the double, adjoint
 * double and single layer forms. Quadrature per element pair: the 7-point rule on both
 * triangles for pairs sharing no vertex; for pairs sharing a vertex (2 regions), an edge (6) or
 * identical (6), each region of a transformation to the unit 4-cube whose Jacobian cancels the
 * 1/r singularity, with 4 Gauss-Legendre points per dimension.
 * The op works with nat_bem_solve (neumann: nt x nrhs, p_out: nv x nrhs, P1 values at the
 * vertices), nat_bem_eval, nat_bem_far_field and nat_bem_sample_field (p: nv x nrhs, neumann:
 * nt x nrhs; the 7-point rule on every element with p interpolated), nat_bem_reassemble, mixed
 * precision, nat_bem_op_apply (R takes nt x nrhs) and nat_bem_op_rows (R rows have nt
 * columns); not with nat_bem_eval_noalloc, nat_bem_run_batch or the server.
 * Arguments as for nat_bem_assemble. Device scratch during assembly: element-pair blocks of
 * rounds of test triangles (about 4 GB, at least 512 triangles x nt x 96 bytes), released
 * before returning.
 * NAT_BEM_EINVAL: as for nat_bem_assemble, a vertex that belongs to no triangle, nt > 65536.
 * NAT_BEM_ENOMEM / NAT_BEM_ECUDA as for nat_bem_assemble.
 */
NAT_BEM_API nat_bem_status nat_bem_assemble_galerkin(const double* verts, int64_t nv, const int32_t* tris,
                                                     int64_t nt, double k, const nat_bem_opts* opts,
                                                     void* cuda_stream, nat_bem_op** out);

/* Number of Neumann values per right-hand side the op takes (columns of R): the triangles of
 * a Galerkin op, else the unknowns (nat_bem_op_size). 0 for NULL. */
NAT_BEM_API int64_t nat_bem_op_neumann_size(const nat_bem_op* op);

/*
 * Monte-Carlo BEM (paper Sec. 4.1.1 "Monte-Carlo-based integration approximation" and Sec. 4.2
 * "Singularity handling"): the conventional boundary integral equation (beta = 0 in Eq. 6)
 * with the surface integral replaced by a sum over m sample points of uniform density on the
 * surface, collocated at the samples. With w = area / m and the sample's own disk of radius
 * eps, pi eps^2 = area / m (single layer over the disk = (eps/2) g_i, double layer 0):
 *
 *   L_ij = 1/2 d_ij - w dG/dn_y(y_i, y_j) (1 - d_ij),   R_ij = -w G(y_i, y_j) (1 - d_ij) - (eps/2) d_ij.
 *
 * The op then works with nat_bem_solve (p at the samples from g at the samples),
 * nat_bem_eval (field = sum_j w [p_j dG/dn_y - g_j G]), nat_bem_reassemble and mixed
 * precision; nat_bem_run_batch and the server take meshes only. The samples are the caller's
 * draw (uniform random or Poisson-disk, Sec. 4.2); the solver does not sample.
 *   pts: m x 3 float64 sample positions; normals: m x 3 float64 unit outward normals
 *   (|n|^2 within 1e-6 of 1); area: total surface area (> 0); host or device pointers.
 * NAT_BEM_EINVAL: out or arrays NULL, m < 2, area or k not positive and finite, a non-finite
 * position, a normal that is not a unit vector. NAT_BEM_ENOMEM / NAT_BEM_ECUDA as for
 * nat_bem_assemble.
 */
NAT_BEM_API nat_bem_status nat_bem_assemble_mc(const double* pts, const double* normals, int64_t m,
                                               double area, double k, const nat_bem_opts* opts,
                                               void* cuda_stream, nat_bem_op** out);

/*
 * Poisson-disk samples of a triangle mesh for nat_bem_assemble_mc (paper Sec. 4.2: samples at
 * a minimum distance cover the surface evenly; the paper samples in parallel on the GPU after
 * Bowers et al. 2010). Dart throwing on a grid, deterministic for given draws:
 *   1. candidate i from draw u_i = (u0, u1, u2): the first triangle whose cumulative area
 *      (FP64, in triangle order) exceeds u0 * total area, at barycentric coordinates
 *      (1 - sqrt(u1), sqrt(u1) (1 - u2), sqrt(u1) u2), with that triangle's unit normal;
 *   2. cells of size h = radius / sqrt(3) over the vertices' bounding box (at most one
 *      sample per cell), cell = floor((x - lo) / h) per axis, clamped;
 *   3. 27 phases (i mod 3, j mod 3, k mod 3) in lexicographic order: each cell of the phase
 *      accepts its lowest-index candidate with no accepted sample closer than radius in the
 *      5 x 5 x 5 cells around it (cells of one phase run in parallel).
 * The accepted candidates come out in increasing index, the same set for any launch order.
 *   verts: nv x 3 float64, tris: nt x 3 int32 (host or device). u: m x 3 float64 draws in
 *   [0, 1) (host or device; the caller's random numbers). idx_out: cap int64 (host, may be
 *   NULL): indices of the accepted candidates. pts_out, normals_out: cap x 3 float64 (host or
 *   device; may be NULL when cap = 0). *count: the number of accepted samples (host), also set
 *   when it exceeds cap (then NAT_BEM_EINVAL and only idx_out's first cap entries are written).
 * Blocks until the outputs are written; m = 0 gives *count = 0.
 * NAT_BEM_EINVAL: NULL arrays, nv or nt < 1, m < 0 or > 2^31 - 1, radius not positive and
 * finite, a triangle index out of range, a degenerate triangle, more than 2^28 grid cells,
 * more samples than cap. NAT_BEM_ENOMEM / NAT_BEM_ECUDA as for nat_bem_assemble.
 */
NAT_BEM_API nat_bem_status nat_bem_poisson_sample(const double* verts, int64_t nv, const int32_t* tris,
                                                  int64_t nt, double radius, const double* u, int64_t m,
                                                  int64_t cap, int64_t* idx_out, double* pts_out,
                                                  double* normals_out, int64_t* count, void* cuda_stream);

/*
 * Re-assembles L and R of an existing op at a new wavenumber k (> 0, finite): the mesh checks,
 * the device geometry, the operator memory and the solver workspace are reused, so sweeping
 * the frequencies of one body costs only the element-pair kernels. Work is ordered on
 * cuda_stream after the op's earlier work on it. NAT_BEM_EINVAL: op NULL or bad k.
 */
NAT_BEM_API nat_bem_status nat_bem_reassemble(nat_bem_op* op, double k, void* cuda_stream);

/*
 * Solves L p = R g for nrhs right-hand sides (GMRES from p = 0, Sec. 6.1 settings by default).
 *   neumann: nt x nrhs complex64, column-major.  p_out: same layout, receives p.
 *   info: may be NULL.  Blocks until the solve is done.
 *   cuda_stream: NULL (the legacy default stream) runs the solve on a stream the op owns,
 *   after the work already queued on the legacy stream (the legacy stream cannot be captured
 *   into the CUDA graphs the solver replays).
 * Convergence: plain FP32, GMRES's residual estimate reaches tol (the true residual with the
 * FP32 operator, reported in info->rel_residual, can sit above tol at high k). Restarted
 * (opts.restart = m > 0): cycles of at most m iterations, each on the true residual with the
 * FP32 operator, until a cycle's estimate or the true residual reaches tol relative to
 * ||R g||, within max_iter iterations in all. Mixed: the true
 * residual reaches tol after a refinement sweep; when a sweep shrinks a residual by less than
 * 10x, or the sweeps or max_iter inner iterations are spent, one final solve of the correction
 * equation on the FP32 operator (its own max_iter) finishes by the plain criterion. A sweep
 * that shrinks a residual by less than 10x with every unconverged true residual within 4 tol
 * ends the solve (the rounding floor of the FP32 residual product; info->rel_residual then
 * reports a value in (tol, 4 tol]).
 * NAT_BEM_EINVAL: op NULL, nrhs < 1, NULL arrays.
 * NAT_BEM_ENOCONV: the tolerance was not met within the iteration limit; p_out holds the
 * best iterate and info is filled.
 */
NAT_BEM_API nat_bem_status nat_bem_solve(nat_bem_op* op, const float* neumann, int32_t nrhs, float* p_out,
                             nat_bem_solve_info* info, void* cuda_stream);

/*
 * Field pressure at m points (paper Sec. 3.4: the pressure anywhere follows from the Neumann and
 * the solved Dirichlet data; this is the exterior representation formula with the Green's
 * function of Sec. 4.2, whose limit on the surface is the first line of Sec. 4, Eq. 6):
 *   field[q, s] = sum_j int_j [p_js dG/dn_y - g_js G](x_q, y) dS_y
 * with the 7-point rule on every element (points should lie off the surface by at least an
 * element size). pts: m x 3 float64.  p, neumann: nt x nrhs complex64 column-major.
 * field_out: m x nrhs complex64 column-major. m = 0 is allowed and does nothing.
 * Returns when the work is enqueued (device outputs) or copied back (host outputs).
 * NAT_BEM_EINVAL: op NULL, m < 0, nrhs < 1, NULL arrays.
 */
NAT_BEM_API nat_bem_status nat_bem_eval(const nat_bem_op* op, const double* pts, int64_t m, const float* p,
                            const float* neumann, int32_t nrhs, float* field_out,
                            void* cuda_stream);

/*
 * nat_bem_eval without any device allocation, for callers that may not allocate device memory
 * (for example code that runs inside another memory manager, under a budget a host framework
 * enforces, or where every device buffer must come from the caller). The paper has no
 * counterpart; it computes exactly what nat_bem_eval computes.
 *   All of pts, p, neumann and field_out must be device pointers (NAT_BEM_EINVAL otherwise):
 *   host staging would allocate. m may be at most 65,536 per call (NAT_BEM_EINVAL with a
 *   message beyond that; split larger point sets over several calls).
 *   Partial sums go to a fixed 4 MiB array compiled into the library, which every GPU that
 *   loads the library holds until the process exits. The first call on each device looks up
 *   that array's device address (make that first call before any stream capture) and keeps
 *   it, so the library must not be used across a cudaDeviceReset. All calls
 *   share the array and it keeps the last call's partial sums, which the next call overwrites
 *   before reading (nothing needs to start at zero); calls that overlap on the GPU (different
 *   streams, or different host threads) race on it and must be serialised by the caller.
 *   Returns when the work is enqueued on cuda_stream.
 */
NAT_BEM_API nat_bem_status nat_bem_eval_noalloc(const nat_bem_op* op, const double* pts, int64_t m,
                                                const float* p, const float* neumann,
                                                int32_t nrhs, float* field_out,
                                                void* cuda_stream);

/*
 * One solve of a batch: the mesh, the wavenumber, the Neumann data (nt x nrhs) and the field
 * points (m x 3, m may be 0) in, the surface pressure (nt x nrhs) and the field (m x nrhs)
 * out, with the job's solve info and status. Arrays follow the conventions above (host or
 * device). Jobs may share a mesh: pass the same verts / tris pointers.
 */
typedef struct {
  const double* verts;
  int64_t nv;
  const int32_t* tris;
  int64_t nt;
  double k;
  const float* neumann;
  int32_t nrhs;
  const double* pts;
  int64_t m;
  float* p_out;
  float* field_out;
  nat_bem_solve_info info; /* out */
  nat_bem_status status;   /* out */
  float device_ms;         /* out: device time from the job's assembly to its field (CUDA events) */
} nat_bem_job;

/*
 * Runs njobs solves (assemble, GMRES, field) with `concurrency` workers (1..32), each on its
 * own stream and op, largest meshes first. A worker that meets the same mesh again re-assembles
 * its op at the new wavenumber (nat_bem_reassemble) instead of rebuilding it. Work starts after
 * the caller's earlier work on cuda_stream; the call returns when every job is done. Returns
 * NAT_BEM_OK when every job succeeded, otherwise the first failing status other than
 * NAT_BEM_ENOCONV if any, else NAT_BEM_ENOCONV; each job's own status is in jobs[i].status.
 */
NAT_BEM_API nat_bem_status nat_bem_run_batch(nat_bem_job* jobs, int32_t njobs,
                                             const nat_bem_opts* opts, int32_t concurrency,
                                             void* cuda_stream);

/*
 * Fused batch (no counterpart in the paper; it batches the per-object solves of the data
 * generation, Sec. 3.4): the jobs' meshes are sorted by size and grouped into buckets of
 * meshes within a factor 2^(1/4) of the bucket's largest triangle count N (at most max_batch
 * meshes, and at most 24 GB of operators per bucket). A bucket is solved as one system of
 * independent operators in lockstep: each mesh's L and R (and BF16 copy) are assembled into
 * one allocation, padded to N unknowns (identity rows in L, zero rows in R and zero right-hand
 * side entries past the mesh's own n, which leaves its solution unchanged), and every GMRES
 * iteration is one matvec launch over all the bucket's operators and one cooperative Arnoldi
 * launch over all its Krylov spaces (captured in CUDA graphs), each mesh with its own
 * convergence test. Each job's field is then evaluated on its own mesh. Jobs with nrhs > 1
 * are solved one after another through the ordinary path. Results match nat_bem_run_batch's to
 * rounding (summation orders differ with the padded size), within the solver's tolerance.
 *   jobs, njobs, opts: as for nat_bem_run_batch (opts NULL = defaults; NAT_BEM_PREC_MIXED_TF32
 *   solves a bucket in plain FP32: its products are matvecs, not GEMMs). max_batch: 1..256.
 *   concurrency: 1..32 host workers, each with its own stream, take the buckets largest first
 *   (then the jobs with several right-hand sides), so one bucket's mesh checks and assembly
 *   overlap another's solve. Work starts after the caller's earlier work on cuda_stream; the
 *   call returns when every job is done, with the statuses and device_ms (the device time of
 *   the job's bucket, assembly to field) filled in.
 * Returns as nat_bem_run_batch does. NAT_BEM_EINVAL: a bad argument (checked for every job
 * before any work), opts out of range.
 */
NAT_BEM_API nat_bem_status nat_bem_run_batch_fused(nat_bem_job* jobs, int32_t njobs,
                                                   const nat_bem_opts* opts, int32_t max_batch,
                                                   int32_t concurrency, void* cuda_stream);

/*
 * Far-field pattern, the leading term Phi_1 of the FFAT expansion |p(x)| = sum_i Phi_i(theta,
 * phi) / r^i (paper Sec. 3.1): for unit directions d_q,
 *   F(d) = lim_{r -> inf} r e^{-ikr} p(r d) = (1/4pi) int [ p (-i k d.n_y) - g ] e^{-ik d.y} dS_y,
 * with the rule of nat_bem_eval (7 points per element; one point of weight area/m per sample
 * for a Monte-Carlo op). |F| over a (theta, phi) grid of directions is the FFAT map (the paper
 * uses 64 x 32, Sec. 5).
 *   dirs: nd x 3 float64 unit vectors.  p, neumann: nt x nrhs complex64 column-major.
 *   out: nd x nrhs complex64 column-major.  Host or device pointers; nd = 0 does nothing.
 * NAT_BEM_EINVAL: op NULL, nd < 0, nrhs < 1, NULL arrays.
 */
NAT_BEM_API nat_bem_status nat_bem_far_field(const nat_bem_op* op, const double* dirs, int64_t nd,
                                             const float* p, const float* neumann, int32_t nrhs,
                                             float* out, void* cuda_stream);

/*
 * Training samples of the neural transfer field (paper Sec. 3.4): n points at spherical
 * coordinates theta = pi u0, phi = 2 pi u1, r = r_lo + (r_hi - r_lo) u2 about `center` (the
 * paper draws them uniformly with r between 1.5 and 3 times the scene's bounding radius), and
 * the pressure amplitude |p| there (the paper trains on the amplitude only).
 *   u: n x 3 float64 draws in [0, 1) (the caller's random numbers).  center: 3 float64 (host).
 *   p, neumann: nt x nrhs complex64.  coords_out: n x 3 float64 (theta, phi, r).
 *   amp_out: n x nrhs float32 column-major.  Host or device pointers; n = 0 does nothing.
 * NAT_BEM_EINVAL: op or center NULL, n < 0, nrhs < 1, NULL arrays, not 0 < r_lo <= r_hi finite.
 */
NAT_BEM_API nat_bem_status nat_bem_sample_field(const nat_bem_op* op, const double* u, int64_t n,
                                                const double* center, double r_lo, double r_hi,
                                                const float* p, const float* neumann, int32_t nrhs,
                                                double* coords_out, float* amp_out, void* cuda_stream);

/*
 * Y = M X with the assembled M = L (which = 0) or R (which = 1) for nrhs complex64 vectors
 * (X, Y: nt x nrhs, column-major; host or device), by the chosen product engine:
 *   NAT_BEM_ENGINE_AUTO: the solver's accurate product (GEMV for one vector, FP32 GEMM else);
 *   NAT_BEM_ENGINE_FP32: FP32 CUDA-core complex GEMM;
 *   NAT_BEM_ENGINE_TF32 / NAT_BEM_ENGINE_BF16 / NAT_BEM_ENGINE_FP16: tcgen05 tensor cores on L
 *     (TF32) or on its BF16 copy (op built with NAT_BEM_PREC_MIXED_BF16) or its row-scaled FP16
 *     copy (NAT_BEM_PREC_MIXED_FP16), FP32 accumulation, nrhs <= 128, L only;
 *   NAT_BEM_ENGINE_GEMV0 + v: GEMV variant v (0 <= v < NAT_BEM_GEMV_VARIANTS; one vector):
 *     0-2 register-tiled (2 or 4 rows per block), 3-4 bulk-copy staged, 5-7 persistent blocks
 *     with x staged in shared memory (plain variant when 8 * ld bytes exceed 200 KiB).
 * This is the operator product of the GMRES iterations (Sec. 4 operators of Eq. 6), exposed
 * for checking and for callers that iterate themselves. Blocks until Y is written.
 * NAT_BEM_EINVAL: bad which / engine / nrhs, engine not usable for this op.
 */
enum {
  NAT_BEM_ENGINE_AUTO = 0,
  NAT_BEM_ENGINE_FP32 = 1,
  NAT_BEM_ENGINE_TF32 = 2,
  NAT_BEM_ENGINE_BF16 = 3,
  NAT_BEM_ENGINE_FP16 = 4,
  NAT_BEM_ENGINE_GEMV0 = 10,
  NAT_BEM_GEMV_VARIANTS = 8
};
NAT_BEM_API nat_bem_status nat_bem_op_apply(const nat_bem_op* op, int32_t which, int32_t engine,
                                            const float* X, int32_t nrhs, float* Y,
                                            void* cuda_stream);

/* The GEMV variant (0 <= v < NAT_BEM_GEMV_VARIANTS) the solver's autotuner chose on the current
 * device for operators of nt elements (sizes are grouped by nt rounded up to 1024), or -1 if
 * no solve of that size has run yet. The tuner times every variant on the operator itself the
 * first time a size is met; NATBEM_GEMV_VARIANT=v in the environment bypasses it. */
NAT_BEM_API int32_t nat_bem_gemv_variant(int64_t nt);

/*
 * Serving (no counterpart in the paper; it serves the data-generation loop of Sec. 3.4). A
 * server runs `slots` workers, each with its own stream. Requests (nat_bem_job, as for the
 * batch driver) are admitted in arrival order as soon as a worker is free and the device
 * bytes the request needs (nat_bem_required_bytes) fit under budget_bytes next to the requests
 * already running; admitted requests overlap on the device. A request that needs more than the
 * whole budget finishes with status NAT_BEM_ENOMEM. The job struct and its arrays must stay
 * valid until nat_bem_wait returns for its ticket. Results do not depend on what else runs:
 * every reduction has a fixed order.
 *   nat_bem_server_create: NAT_BEM_EINVAL (budget <= 0, slots not in 1..64), NAT_BEM_ECUDA
 *     (no device). With the environment variable NATBEM_SERVER_FAKE=1 the workers do no device
 *     work (a request "takes" nt x 10 us and succeeds): a mode for testing the host logic.
 *   nat_bem_submit: enqueue; *ticket identifies the request. NAT_BEM_EBUSY after destroy began.
 *   nat_bem_wait: waits up to timeout_ms (< 0: forever) and returns the request's status, or
 *     NAT_BEM_ETIMEOUT (the request stays queued; wait again). queue_ms / total_ms (may be
 *     NULL): host time from submit to admission and to completion.
 *   nat_bem_server_reserved: device bytes reserved by running requests.
 *   nat_bem_server_destroy: finishes queued and running requests, then stops the workers.
 */
typedef struct nat_bem_server nat_bem_server;
NAT_BEM_API nat_bem_status nat_bem_server_create(int64_t budget_bytes, const nat_bem_opts* opts,
                                                 int32_t slots, nat_bem_server** out);
NAT_BEM_API nat_bem_status nat_bem_submit(nat_bem_server* srv, nat_bem_job* job, int64_t* ticket);
NAT_BEM_API nat_bem_status nat_bem_wait(nat_bem_server* srv, int64_t ticket, int32_t timeout_ms,
                                        double* queue_ms, double* total_ms);
NAT_BEM_API int64_t nat_bem_server_reserved(nat_bem_server* srv);
NAT_BEM_API void nat_bem_server_destroy(nat_bem_server* srv);

/*
 * Self-test of the bounded device waits (no counterpart in the paper). A kernel waits on an
 * mbarrier that nothing ever completes, with the same bounded-wait code the tensor-core and
 * bulk-copy kernels use but a deadline of timeout_ms (1..10000); it must give up, report it
 * through a device flag and return. Returns NAT_BEM_ETIMEOUT when it did (the expected
 * result; the CUDA context stays usable), NAT_BEM_OK if the wait completed (never expected),
 * NAT_BEM_EINVAL for a bad timeout, NAT_BEM_ECUDA for a CUDA failure. Blocks until done.
 */
NAT_BEM_API nat_bem_status nat_bem_selftest_bounded_wait(int32_t timeout_ms, void* cuda_stream);

/*
 * Copies rows [row0, row0 + nrows) of the assembled L (which = 0) or R (which = 1) into
 * out (nrows x cols complex64, row-major; cols = nat_bem_op_size for L,
 * nat_bem_op_neumann_size for R). For checking the operator; not on the solve path.
 * NAT_BEM_EINVAL: rows out of range, which not 0/1, R not stored.
 */
NAT_BEM_API nat_bem_status nat_bem_op_rows(const nat_bem_op* op, int32_t which, int64_t row0, int64_t nrows,
                               float* out, void* cuda_stream);

/* Number of unknowns of the op: triangles (nat_bem_assemble), samples (nat_bem_assemble_mc)
 * or vertices (nat_bem_assemble_galerkin); 0 for NULL. */
NAT_BEM_API int64_t nat_bem_op_size(const nat_bem_op* op);

/* Device bytes an op of nt triangles with nrhs right-hand sides holds under opts (NULL =
 * defaults): the operators plus the solver workspace. Used for admission control. */
NAT_BEM_API int64_t nat_bem_required_bytes(int64_t nt, int32_t nrhs, const nat_bem_opts* opts);

/* Frees the op and its device memory (stream-ordered on the stream it was built on). NULL ok. */
NAT_BEM_API void nat_bem_destroy(nat_bem_op* op);

/*
 * Tracing for benchmarks and profiling (no counterpart in the paper). Every kernel launch of
 * the library is counted. With tracing enabled, each launch is also bracketed by two CUDA
 * events recorded on its stream; nat_bem_trace_kernel waits for the recorded events and
 * returns the summed device time and the number of launches of the kernels whose name contains
 * `name` ("" = all). Names: "assemble_regular", "assemble_near", "geometry", "gemv",
 * "gmres_dots", "gmres_update_dots", "gmres_update_norm", "gmres_normalize", "eval", ...
 * The counters are process-wide and not thread-safe against concurrent resets.
 */
NAT_BEM_API void nat_bem_trace_enable(int32_t enable);
/* With tracing enabled, record events only for kernels whose name contains one of the
 * comma-separated substrings in `names` (NULL or "" = every kernel). */
NAT_BEM_API void nat_bem_trace_select(const char* names);
NAT_BEM_API void nat_bem_trace_reset(void);
NAT_BEM_API int64_t nat_bem_trace_launches(void);
NAT_BEM_API nat_bem_status nat_bem_trace_kernel(const char* name, double* total_ms,
                                                int64_t* launches);
/* Per-launch device times (ms, in launch order) of the traced kernels named exactly `name`:
 * the first min(cap, count) go to out_ms, *count receives how many there are. Lets a caller
 * tell launches that did work from those that exited at once (a GMRES iteration of a captured
 * chunk after convergence). NAT_BEM_EINVAL: name NULL, cap < 0, out_ms NULL with cap > 0. */
NAT_BEM_API nat_bem_status nat_bem_trace_durations(const char* name, float* out_ms, int64_t cap,
                                                   int64_t* count);

/*
 * Neural acoustic transfer field (Sec. 3.3, Eq. 3 and 4; Sec. 3.4): the learned map from the
 * spherical coordinates of a listening point, the condition variables and the frequency to the
 * outputs (one per mode, or one pressure amplitude). One forward pass per query:
 *   inputs  x = (theta/pi, phi/(2 pi), r_norm, v_1..v_c, f), D = 4 + n_cond values in [0, 1];
 *   grid    4 levels of 8, 16, 32, 64 cells per axis over (x_0, x_1, x_2), 4 features per
 *           vertex, trilinear interpolation; a level with (N + 1)^3 <= 2^table_log2 vertices is
 *           dense (row i + (N + 1)(j + (N + 1) k)), a finer one hashed: row
 *           (i xor j * 2654435761 xor k * 805459861) mod 2^table_log2 (32-bit arithmetic);
 *   PE      sin and cos of 2^l pi x_d, l = 0..5, for d = 3..D-1 (v, then f), ordered (d, l,
 *           sin/cos);
 *   MLP     [16 grid features, PE, zeros] (128 wide) -> 4 x (128, ReLU) -> n_out, linear.
 * The layers run on the tensor cores with BF16 weights and BF16 layer inputs (each layer's
 * input is rounded to nearest-even BF16) and FP32 accumulation, bias and output.
 *
 * nat_field_create copies the parameters to the device of the current context (host or device
 * pointers; the caller keeps ownership of its arrays):
 *   tables  float32, the four levels' rows one level after the other, 4 features per row;
 *           level l has min((N_l + 1)^3, 2^table_log2) rows. The field keeps them in half
 *           precision (rounded to nearest, as tiny-cuda-nn stores grid parameters);
 *   weights float32, row-major [out][in]: four 128 x 128 hidden layers, then the n_out x 128
 *           output layer. The field keeps them in BF16 (rounded to nearest-even on creation);
 *   biases  float32: 4 x 128, then n_out.
 *   NAT_BEM_EINVAL: NULL argument, n_cond not in 0..8, n_out not in 1..128, table_log2 not in
 *   12..24. NAT_BEM_ENOMEM / NAT_BEM_ECUDA: device allocation or copy failed.
 * nat_field_forward: x n x D float32 row-major, out n x n_out float32 row-major, host or device
 *   pointers, on cuda_stream; blocks until out is written; n = 0 does nothing. With a host x or
 *   out and n > 2^20, the queries go in chunks of 2^20 whose uploads and downloads (on two copy
 *   streams the field keeps) overlap the other chunks' kernels; pinned host memory makes the
 *   copies asynchronous. Calls on one field must not run concurrently. NAT_BEM_EINVAL for NULL
 *   or n < 0; NAT_BEM_ETIMEOUT if a bounded wait on the tensor cores gave up (the output is
 *   then incomplete).
 * nat_field_destroy frees the device copies (NULL is a no-op).
 */
typedef struct nat_field nat_field;
NAT_BEM_API nat_bem_status nat_field_create(int32_t n_cond, int32_t n_out, int32_t table_log2,
                                            const float* tables, const float* weights,
                                            const float* biases, void* cuda_stream, nat_field** out);
NAT_BEM_API nat_bem_status nat_field_forward(const nat_field* f, const float* x, int64_t n,
                                             float* out, void* cuda_stream);
NAT_BEM_API void nat_field_destroy(nat_field* f);

/* Message of the last failed call on this thread ("" if none). */
NAT_BEM_API const char* nat_bem_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* NAT_BEM_H */
