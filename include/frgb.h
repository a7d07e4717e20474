/* frgb -- Flux Reconstruction right-hand side on one GB300 GPU.
 *
 * C ABI of the library.  It evaluates the right-hand side of the
 * Flux Reconstruction (FR) discretisation of the compressible Euler and
 * Navier-Stokes equations (PyFR v2.0.3, arXiv 2408.16509, Section 2) on
 * meshes of linear hexahedra, prisms and tetrahedra, and advances it with
 * explicit Runge-Kutta schemes.  Every step of the right-hand side runs in
 * the library's CUDA kernels (sm_103a); there is no CPU fallback.
 *
 * Conventions shared by all calls
 *   - Return value: FR_OK (0) on success, a negative FR_E* code otherwise;
 *     fr_last_error() gives a message for the calling thread.
 *   - The library copies every host input; the caller keeps ownership of
 *     its buffers.  Handles are opaque and released by fr_mesh_destroy.
 *   - Host solution layout: per element type, [n_elem][nupts][5], FP64,
 *     variables (rho, rho u, rho v, rho w, E); point order as returned by
 *     fr_get_points.
 *   - Element vertex order (reference coordinates of each vertex):
 *       FR_HEX8: (-1,-1,-1) (1,-1,-1) (1,1,-1) (-1,1,-1)
 *                (-1,-1, 1) (1,-1, 1) (1,1, 1) (-1,1, 1)
 *       FR_PRI6: (-1,-1,-1) (1,-1,-1) (-1,1,-1) (-1,-1,1) (1,-1,1) (-1,1,1)
 *       FR_TET4: (-1,-1,-1) (1,-1,-1) (-1,1,-1) (-1,-1,1)
 *     Elements must be positively oriented (det J > 0 everywhere).
 *   - Calls on one handle are not thread-safe; kernels run on the handle's
 *     stream (fr_set_stream).
 */
#ifndef FRGB_H
#define FRGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FR_OK = 0,
  FR_EINVAL = -1,      /* bad argument */
  FR_ENOMEM = -2,      /* device or host allocation failed */
  FR_ECUDA = -3,       /* a CUDA call failed (message has the CUDA error) */
  FR_EMESH = -4,       /* non-conforming mesh, unmatched face, bad Jacobian */
  FR_ENONFINITE = -5,  /* a right-hand side produced NaN or Inf */
  FR_EFILTER = -6,     /* entropy-filter root-find fell back to bisection */
  FR_ETIMEOUT = -7     /* a bounded device wait expired */
};

enum { FR_HEX8 = 0, FR_PRI6 = 1, FR_TET4 = 2 };
enum { FR_EULER = 0, FR_NAVIER_STOKES = 1 };
/* FR_FP64: everything in FP64.  FR_FP32: everything in FP32.
 * FR_MIXED: traces, fluxes, operators and stage values in FP32, the RK
 * solution and accumulator registers in FP64 (hexahedral meshes). */
enum { FR_FP64 = 0, FR_FP32 = 1, FR_MIXED = 2 };
enum { FR_BC_STATE = 0, FR_BC_EXTRAPOLATE = 1, FR_BC_EXCHANGE = 2, FR_BC_PRESCRIBED = 3 };
enum { FR_RK4 = 0, FR_RK45 = 1 };
/* Line points of hexahedra (fr_mesh_desc.point_family). */
enum { FR_POINTS_GL = 0, FR_POINTS_GLL = 1 };

typedef struct fr_mesh fr_mesh;
typedef struct fr_group fr_group;

typedef struct {
  int etype;            /* FR_HEX8, FR_PRI6 or FR_TET4 */
  int64_t n_elem;
  const int64_t* conn;  /* [n_elem][n_vertices] node ids (face pairing; and
                           the map of straight elements) */
  int map_order;        /* 0 or 1: straight elements (vertex map); 2:
                           quadratic map, 3: cubic map (Section 3.4
                           "Curved Elements") given by map_conn */
  const int64_t* map_conn;  /* map_order 2 or 3: [n_elem][n_map] node ids of
                               the map; its vertex nodes must be the vertices
                               of conn.
                               FR_HEX8, order 2, 27 nodes: node a + 3b + 9c at
                               reference point (-1+a, -1+b, -1+c); order 3,
                               64 nodes: node a + 4b + 16c at
                               (-1+2a/3, -1+2b/3, -1+2c/3);
                               FR_PRI6, 18 nodes: triangle node + 6 layer,
                               triangle nodes v0, v1, v2 and the midpoints of
                               edges 01, 12, 02, layers z = -1, 0, 1 (the
                               vertices are nodes 0, 1, 2, 12, 13, 14);
                               FR_TET4, 10 nodes: v0..v3, then the midpoints
                               of edges 01, 12, 02, 03, 13, 23.
                               Order 3: FR_PRI6, 40 nodes: triangle node +
                               10 layer, layers z = -1, -1/3, 1/3, 1,
                               triangle nodes v0, v1, v2, two on each of the
                               edges 01, 12, 02 (at 1/3 then 2/3 of the way
                               from the edge's first vertex) and the
                               centroid (the vertices are nodes 0, 1, 2, 30,
                               31, 32); FR_TET4, 20 nodes: v0..v3, two on
                               each of the edges 01, 12, 02, 03, 13, 23 (in
                               the same way), the centroids of the faces 012,
                               013, 023, 123.
                               Metrics of curved elements: the conservative
                               curl form S[i][n] = -(curl I(X_l grad X_m))_i,
                               I the order-p interpolant on nodes with nodes
                               on every face (Gauss-Lobatto tensor nodes,
                               warp-and-blend tetrahedron nodes, the
                               tetrahedron's face nodes times Gauss-Lobatto
                               points for prisms) */
} fr_etype_desc;

typedef struct {
  int tag;              /* boundary-face tag this condition applies to */
  int kind;             /* FR_BC_PRESCRIBED: outside state given point by
                           point by the caller (fr_set_bc_state; state[]
                           unused); FR_BC_EXCHANGE: a face between parts of a
                           partitioned mesh, its outside state the partner
                           part's (meshes with such faces run only in a
                           group, fr_group_create); FR_BC_STATE: outside
                           state = state (primitive
                           rho, u, v, w, p); FR_BC_EXTRAPOLATE: outside
                           state = inside state */
  double state[5];
} fr_bc_desc;

typedef struct {
  int64_t n_nodes;
  const double* nodes;            /* [n_nodes][3] */
  int n_etypes;
  const fr_etype_desc* etypes;    /* at most one entry per element type */
  int order;                      /* polynomial order p, 1..4 */
  int physics;                    /* FR_EULER or FR_NAVIER_STOKES */
  double gamma, mu, prandtl;      /* ratio of specific heats, dynamic
                                     viscosity (constant), Prandtl number */
  int n_periodic;                 /* 0..3 translation vectors */
  double periodic[3][3];
  int64_t n_bfaces;
  const int64_t* bface_nodes;     /* [n_bfaces][4] node ids, -1 pads tris */
  const int* bface_tags;          /* [n_bfaces] */
  int n_bcs;                      /* <= 8 */
  const fr_bc_desc* bcs;
  int precision;                  /* FR_FP64, FR_FP32 or FR_MIXED */
  int device;                     /* CUDA device ordinal; < 0 builds a
                                     host-only handle (geometry, points and
                                     operators; no GPU is touched and the
                                     compute calls return FR_EINVAL) */
  int point_family;               /* hexahedra: FR_POINTS_GL (0, default)
                                     Gauss-Legendre solution and flux
                                     points; FR_POINTS_GLL Gauss-Lobatto
                                     solution points with the flux points
                                     among them, so the interpolation of
                                     Eq. (disu) is a gather (Section 3.1,
                                     "Matrix multiplications", last
                                     paragraph).  GLL needs a mesh without
                                     prisms (FR_EINVAL): their quad faces
                                     carry Gauss-Legendre points */
} fr_mesh_desc;

/* Build a discretisation (Section 2: conforming tessellation, reference
 * mappings, solution and flux points).  Faces are paired by their vertex
 * sets, then periodically by translated centroids; every remaining face
 * must be listed in bface_nodes.  Flux points are paired by physical
 * coordinates.  FR_EMESH: non-conforming or unmatched faces, det J <= 0.
 * Allocates device memory (all state lives on device `device`). */
int fr_mesh_create(const fr_mesh_desc* desc, fr_mesh** out);

/* Release all host and device memory of the handle.  NULL is allowed. */
int fr_mesh_destroy(fr_mesh* mesh);

/* Element count, solution points and flux points per element of `etype`
 * (zeros when the mesh has no element of that type). */
int fr_get_info(const fr_mesh* mesh, int etype, int64_t* n_elem, int* nupts,
                int* nfpts);

/* Physical coordinates of the solution points: host [n_elem][nupts][3]. */
int fr_get_points(const fr_mesh* mesh, int etype, double* xyz);

/* Copy a solution in (host FP64 [n_elem][nupts][5]) / out. */
int fr_set_solution(fr_mesh* mesh, int etype, const double* u);
int fr_get_solution(const fr_mesh* mesh, int etype, double* u);

/* Allocation-free variant of fr_set_solution (the paper has no
 * counterpart; it serves callers that cannot allocate device memory, such
 * as applications whose device memory is reserved up front by their own
 * pool allocator, or time-stepping loops that must not pay the device-wide
 * synchronisation cudaMalloc / cudaFree can imply).  It calls no
 * cudaMalloc, cudaFree or allocating library routine: the host array is
 * copied into a fixed staging array compiled into the library (16 MiB,
 * i.e. at most 2^21 FP64 values = n_elem * nupts * 5, held by every GPU that
 * loads the library until process exit), then the layout kernel writes the
 * solution register.  Larger solutions return FR_EINVAL.  The first call on
 * a device looks up the array's device address (with that device current)
 * and caches it; make that first call before any stream capture.  All calls
 * share the one staging array, which keeps the last call's contents: calls
 * that overlap on the GPU (e.g. two handles on different streams) race.
 * Synchronous: returns after the copy and the layout kernel completed. */
int fr_set_solution_static(fr_mesh* mesh, int etype, const double* u);

/* Element type of a caller's device array (fr_set_solution_device,
 * fr_get_solution_device). */
enum { FR_DTYPE_F64 = 0, FR_DTYPE_F32 = 1 };

/* Same from / to device memory (e.g. a torch tensor's data pointer) in the
 * host layout [n_elem][nupts][5], element type `dtype` (FR_DTYPE_F64 or
 * FR_DTYPE_F32; values are converted to the handle's register precision),
 * on the handle's stream: asynchronous, the pointer must stay valid until
 * the stream reaches the copy (fr_sync).  FR_EINVAL for another dtype. */
int fr_set_solution_device(fr_mesh* mesh, int etype, const void* dptr, int dtype);
int fr_get_solution_device(const fr_mesh* mesh, int etype, void* dptr, int dtype);

/* Outside state of an FR_BC_PRESCRIBED condition (the prescribed-state
 * boundary of Section 2's problem statement: the outside state u+ of
 * Eq. comm_flux comes from the boundary).  The library calls
 *   fn(n, x, t, prim, ctx)
 * once with the n boundary flux points of condition `tag` (x [n][3], in
 * fr_get_boundary_points order) and time t; fn writes the primitive state
 * prim [n][5] (rho, u, v, w, p) at each.  The states are kept on the device
 * and used by every later right-hand side and RK stage until the next call
 * (a time-dependent condition is updated by the caller, e.g. once per
 * step).  With Navier-Stokes the outside gradient is the inside one, as for
 * FR_BC_STATE.  Compute calls on a mesh with a prescribed condition that
 * has no state yet return FR_EINVAL; so does a non-positive density or
 * pressure.  Synchronous. */
typedef void (*fr_bc_fn)(int64_t n, const double* x, double t, double* prim, void* ctx);
int fr_set_bc_state(fr_mesh* mesh, int tag, fr_bc_fn fn, double t, void* ctx);

/* One evaluation of the right-hand side du/dt = -J^{-1} div~ f~ (Section 2:
 * Eq. disu, interpolation to the flux points; Eq. comm_flux, the common
 * interface flux; Eq. FRfinal, the corrected divergence) at the current
 * solution, for time t.  The boundary conditions of this library do not
 * depend on time, so t only labels the evaluation (fr_stats reports it);
 * t must be finite.  Outputs, either or both may be NULL:
 *   rhs_host: host FP64, all element types in mesh order (hexahedra,
 *             prisms, tetrahedra present), each [n_elem][nupts][5]
 *             concatenated; filled before the call returns;
 *   rhs_dev:  device FP64, same layout; written on the handle's stream.
 * The result also stays on the device for fr_get_rhs (host, one type).
 * FR_ENONFINITE when any entry is NaN or Inf. */
int fr_rhs(fr_mesh* mesh, double t, double* rhs_host, void* rhs_dev);
int fr_get_rhs(const fr_mesh* mesh, int etype, double* rhs);

/* Advance the solution by `nsteps` explicit steps of size dt (Section 2,
 * "a suitable explicit time integration scheme"; Section 3.5 low-storage
 * pairs): FR_RK4 classical four-stage, FR_RK45 the two-register
 * RK4(3)5[2R+]C of Kennedy, Carpenter & Lewis.  One step is replayed as one
 * CUDA graph.  Returns FR_ENONFINITE if any stage produced NaN/Inf. */
int fr_rk_step(fr_mesh* mesh, int scheme, double dt, int nsteps);

/* Adaptive time stepping (Section 3.5, low-storage RK with an embedded
 * pair).  One attempted FR_RK45 step of size *dt: the embedded third-order
 * weights bhat give the error estimate e = dt sum_i (b_i - bhat_i) k_i; its
 * norm err = sqrt(mean_c (e_c / (atol + rtol max(|u^n_c|, |u^{n+1}_c|)))^2)
 * over every component c of every element decides acceptance (err <= 1; a
 * rejected step restores u^n).  *dt receives the next step size from a PI
 * controller: accepted steps dt * clip(0.9 err^-0.175 err_prev^0.1, 0.2, 5)
 * (at most dt right after a rejection), rejected ones
 * dt * max(0.2, 0.9 err^-0.25).  The controller state is the caller's
 * (`ctl`: set atol, rtol; start with err_prev = 1, after_reject = 0).  A
 * stage that produces NaN/Inf counts as a rejection (err = +inf).  Not
 * available with the entropy filter (FR_EINVAL). */
typedef struct {
  double atol, rtol;  /* tolerances of the error norm */
  double err_prev;    /* norm of the last accepted step (controller memory) */
  int after_reject;   /* 1 when the previous attempt was rejected */
} fr_adapt_t;
int fr_rk_adaptive_step(fr_mesh* mesh, fr_adapt_t* ctl, double* dt, int* accepted,
                        double* err);

/* Measurement aid: advances the solution by ONE step of `scheme` exactly
 * as fr_rk_step does, but launches the kernels one by one (no graph) with
 * CUDA events around every launch on the handle's stream.  On return
 * ms[k] holds the summed device time (milliseconds) and launches[k] the
 * launch count of kernel class k during that step, for k < FR_KC_COUNT. */
enum { FR_KC_FACE_U = 0,  /* NS common solution at interior flux points */
       FR_KC_BND_U = 1,   /* NS common solution at boundary flux points */
       FR_KC_GRAD = 2,    /* NS corrected gradients (one launch per type) */
       FR_KC_FACE_F = 3,  /* common normal flux, interior pairs */
       FR_KC_BND_F = 4,   /* common normal flux, boundary points */
       FR_KC_VOL = 5,     /* volume: flux, divergence, lift, RK update */
       FR_KC_FILTER = 6,  /* entropy minimum and entropy filter */
       FR_KC_AAFLUX = 7,  /* anti-aliased transformed flux (one per type) */
       FR_KC_COUNT = 8 };
int fr_profile_step(fr_mesh* mesh, int scheme, double dt, double* ms,
                    int* launches);

/* Counters and timings of a handle (Section 3.1, "Task graphs": what a
 * step costs; Section 3.2, "Entropy filtering": how many elements were
 * filtered and how many margin evaluations the iterative strength search
 * took).  ms_device sums the device time of fr_rhs, fr_rk_step and
 * fr_rk_adaptive_step calls (a pair of CUDA events around each on the
 * handle's stream; none while that stream is being captured); ms_kernel and
 * launches are those of the last fr_profile_step.  fr_stats waits for the
 * timed calls still in flight.  reset != 0 zeroes the counters, the device
 * time and the filter counters after reading them.  Works on host-only
 * handles (all zero). */
typedef struct {
  uint64_t rhs_calls;        /* fr_rhs evaluations */
  uint64_t rk_steps;         /* fixed-size RK steps (fr_rk_step, fr_profile_step) */
  uint64_t rk_attempts;      /* adaptive attempts (fr_rk_adaptive_step) */
  uint64_t rk_rejected;      /*   of which rejected */
  uint64_t stages;           /* right-hand-side evaluations of all of these */
  uint64_t filtered;         /* entropy filter: filtered element-stages */
  uint64_t filter_evals;     /*   margin evaluations (root-find iterations) */
  uint64_t filter_fallbacks; /*   elements left infeasible at zeta = 36 */
  uint64_t predictor_used;   /*   element-stages opened from the predictor */
  double ms_device;          /* device milliseconds of the timed calls */
  double ms_kernel[FR_KC_COUNT];  /* last fr_profile_step, per kernel class */
  int launches[FR_KC_COUNT];
  int kernel_family;         /* FR_VARIANT_* in use */
  double t_last;             /* t of the last fr_rhs */
} fr_stats_t;
int fr_stats(fr_mesh* mesh, fr_stats_t* out, int reset);

/* Kernel family.  For hexahedra: FR_VARIANT_SUMFACT applies the operators
 * line by line (1D factors of the tensor-product basis) with metric terms
 * stored per solution point; FR_VARIANT_SUMFACT_VERTEX (FP32 values only)
 * computes the metric terms from the 8 vertices and recomputes gradients
 * instead of storing them (less DRAM traffic, more arithmetic);
 * FR_VARIANT_DENSE applies the full operator matrices as for prisms and
 * tetrahedra.  FR_VARIANT_TENSOR (FP32 values; prisms and tetrahedra of
 * order 2..3, tetrahedra of order 4): hexahedra as FR_VARIANT_SUMFACT,
 * and the dense operator products of prisms and tetrahedra (Eqs. disu,
 * FRfinal and the gradient path) on the tensor cores as three TF32 products
 * per product (operands split into TF32 hi + lo parts, FP32 accumulation);
 * types without that form keep the CUDA-core kernels.  The other families run
 * prisms and tetrahedra on the CUDA cores.  All give the same result up to
 * rounding.  FR_VARIANT_AUTO (default): the first fr_rk_step times one step
 * of each applicable family on a copy of the state (restored afterwards) and
 * keeps the fastest; fr_get_tuning reports the choice. */
enum { FR_VARIANT_AUTO = 0, FR_VARIANT_DENSE = 1, FR_VARIANT_SUMFACT = 2,
       FR_VARIANT_SUMFACT_VERTEX = 3, FR_VARIANT_TENSOR = 4 };
int fr_set_kernel_variant(fr_mesh* mesh, int variant);

/* Kernel family in use and the step times (ms, 0 if not tried) the tuner
 * measured, ms_per_step[5] indexed by FR_VARIANT_* (entry 0 unused). */
int fr_get_tuning(const fr_mesh* mesh, int* active, float* ms_per_step);

/* Tiles and schedule of the kernels (Section 3.1, "Matrix
 * multiplications": configurations benchmarked at run time, the fastest
 * kept; "Task graphs": independent kernels run in parallel).  Indexed by
 * element kind (FR_HEX8, FR_PRI6, FR_TET4):
 *   tile_grad, tile_vol: gradient / volume kernel tile: elements per CTA of
 *     the sum-factorised hexahedron kernels (at most 256 threads per CTA),
 *     persistent CTAs per SM of the dense kernels; 0 = the largest (default),
 *     -1 = no such element in the mesh;
 *   tensor_grad, tensor_vol: 1 when that kernel runs on the tensor cores;
 *   structured: 1 when the CUDA-core kernels of that kind use the
 *     structure of its operators (Section 3.1, "Matrix multiplications":
 *     sum factorisation on hexahedra; on prisms the triangle x line
 *     factorisation of the derivatives and the nonzeros of the
 *     interpolation and lift; on tetrahedra the interpolation to the flux
 *     points by its nonzeros, a gather), 0 for the dense operator products.
 * face_block: threads per CTA of the interface and boundary kernels (32..1024,
 * a multiple of 32); parallel_types: the per-type kernels of a phase run as
 * parallel branches of the step's graph (forked streams) instead of in
 * order.  ms_default / ms_tuned: step time of the picked family with the
 * default and the tuned schedule (0 until the autotuner ran).  With
 * FR_VARIANT_AUTO the first fr_rk_step tunes all of it after picking the
 * family; every schedule gives the same results bit for bit. */
typedef struct {
  int tile_grad[3], tile_vol[3];
  int tensor_grad[3], tensor_vol[3];
  int face_block;
  int parallel_types;
  float ms_default, ms_tuned;
  int structured[3];
} fr_schedule_t;
int fr_get_schedule(const fr_mesh* mesh, fr_schedule_t* out);
/* Set the tiles and schedule (tensor_*, structured and ms_* are ignored);
 * FR_EINVAL for a tile above the kernel's maximum, a bad block size, or a
 * host-only handle.  Later steps rebuild their graphs. */
int fr_set_schedule(fr_mesh* mesh, const fr_schedule_t* in);

/* Kernels and copies of the handle run on this stream (cudaStream_t);
 * NULL selects the handle's own stream. */
int fr_set_stream(fr_mesh* mesh, void* cuda_stream);

/* Synchronise the handle's stream. */
int fr_sync(fr_mesh* mesh);

/* Reference-element data of `etype`, FP64, host memory, as built by the
 * library (Section 2):
 *   FR_OP_M0      [nfpts][nupts]        l_z(x_f), Eq. (disu)
 *   FR_OP_D       [3][nupts][nupts]     d l_v / d x~_d at x_z, Eq. (FRfinal)
 *   FR_OP_LIFT    [nupts][nfpts]        div~ g_f at x_z (DG correction)
 *   FR_OP_WEIGHTS [nupts]               int l_z over the reference element
 *   FR_OP_UPTS    [nupts][3]            reference solution points
 *   FR_OP_FPTS    [nfpts][3]            reference flux points
 * With anti-aliasing on (fr_set_antialias, degree qdeg; nq = (qdeg/2+1)^3
 * quadrature points on every element type), else FR_EINVAL:
 *   FR_OP_AA_QPTS [nq][3]               quadrature points
 *   FR_OP_AA_QWTS [nq]                  quadrature weights
 *   FR_OP_AA_B    [nq][nupts]           l_z(x_q), solution -> quadrature points
 *   FR_OP_AA_P    [nupts][nq]           least-squares projection back
 * Works on host-only handles too. */
enum { FR_OP_M0 = 0, FR_OP_D = 1, FR_OP_LIFT = 2, FR_OP_WEIGHTS = 3,
       FR_OP_UPTS = 4, FR_OP_FPTS = 5, FR_OP_AA_QPTS = 6, FR_OP_AA_QWTS = 7,
       FR_OP_AA_B = 8, FR_OP_AA_P = 9 };
int fr_get_operator(const fr_mesh* mesh, int etype, int which, double* out);

/* ---------------------------------------------------------------------------
 * Domain decomposition (Section 3.3, "Mixed Elements and Domain Decomposition").
 * Elements carry a global index: the element types in the order hexahedra,
 * prisms, tetrahedra (those present), then the element number.  All three
 * calls work on host-only handles.
 *
 * fr_get_adjacency: nbr [n_elem of etype][n_faces]: global index of the
 * element across each face (periodic partners included), -1 on a boundary.
 *
 * fr_partition: part [total elements] in 0..nparts-1, by recursive
 * coordinate bisection of element centroids.  mode 0 (weighted): element of
 * type k weighs weights[k] (null: all 1); mode 1 (balanced): each type is
 * bisected on its own, so every part holds the same number of elements of
 * each type (to within one) whatever their relative cost.  FR_EINVAL for
 * nparts < 1, another mode or a non-positive weight.
 *
 * fr_partition_faces: the faces of part `rank`'s elements whose neighbour
 * lies in another part, as [count][4] node ids (-1 pads triangles); with
 * faces = null only count is returned.  A sub-mesh of that part lists them
 * as boundary faces with an FR_BC_EXCHANGE condition. */
int fr_get_adjacency(const fr_mesh* mesh, int etype, int64_t* nbr);
/* Boundary flux points in the library's order (count: n_boundary of
 * fr_get_pairs): physical position x [n][3] and condition kind [n]
 * (FR_BC_*); either pointer may be null. */
int fr_get_boundary_points(const fr_mesh* mesh, double* x, int* kind);
/* Interior flux-point pairs in the library's order (count: n_interior of
 * fr_get_pairs): global element index of the "-" (left) and "+" (right)
 * side of each; left <= right by the orientation rule of
 * fr_set_viscous_scheme.  Either pointer may be null. */
int fr_get_interfaces(const fr_mesh* mesh, int64_t* left, int64_t* right);
int fr_partition(const fr_mesh* mesh, int nparts, int mode, const double* weights,
                 int32_t* part);
int fr_partition_faces(const fr_mesh* mesh, const int32_t* part, int rank,
                       int64_t* faces, int64_t* count);

/* Partition groups (the exchange between partitions of Section 3.1,
 * "Multi-node capabilities", here between the parts of a mesh on one
 * device): the parts of one mesh (each created from its elements,
 * with its faces towards other parts as FR_BC_EXCHANGE boundary faces) run
 * together on one device.  fr_group_create matches every exchange flux
 * point with exactly one exchange point of another member by physical
 * position (the members' common periodic translations included); FR_EMESH
 * if a point has no partner or several.  Members must share device,
 * precision, physics, order, constants and periodic vectors, must not run
 * the entropy filter, and must outlive the group; each keeps its own
 * solution (fr_set_solution / fr_get_solution / fr_get_rhs on the member).
 * fr_group_rhs and fr_group_rk_step evaluate the right-hand side / advance
 * all members: at each coupling point of a stage (solution traces before
 * the common solution and fluxes; for Navier-Stokes the gradient traces, or
 * with FP32 values the viscous normal fluxes, before the common fluxes) each
 * member pushes its traces into the partners' receive buffers on the
 * device, then the stage continues, so the result is the unpartitioned
 * mesh's up to rounding.  Runs on the first member's stream and
 * synchronises it.  fr_rhs / fr_rk_step on a member outside its group
 * return FR_EINVAL, and so does fr_mesh_destroy of a member (the mesh is
 * kept) until its group is destroyed. */
int fr_group_create(fr_mesh* const* meshes, int n, fr_group** out);
int fr_group_destroy(fr_group* group);
int fr_group_rhs(fr_group* group);
int fr_group_rk_step(fr_group* group, int scheme, double dt, int nsteps);

/* Exchange between processes (Section 3.1, "Multi-node capabilities": the
 * packed face buffers of the partitions exchanged by MPI; here any transport
 * the caller has, e.g. torch.distributed over gloo or NCCL).  A part of a
 * partitioned mesh, built with its faces towards other parts as
 * FR_BC_EXCHANGE boundaries, lives in its own process (one GPU each):
 *
 * fr_exchange_faces: this part's exchange faces in the library's order,
 *   for the other ranks: n_faces, n_points, and (arrays may be NULL to query
 *   the counts) face_npts [n_faces] points per face, centroids
 *   [n_faces][3], pt_x [n_points][3] positions and pt_mag [n_points] face
 *   metric magnitudes |S^T n~| of the points, face by face.  Host-only
 *   handles too.
 * fr_exchange_setup: match this part's exchange points (rank `rank` of
 *   nranks) with the other ranks' from all ranks' fr_exchange_faces arrays,
 *   concatenated in rank order (faces_per_rank, points_per_rank [nranks]);
 *   faces by translated centroid (the mesh's periodic vectors), then points
 *   by position.  counts [nranks] receives the number of points exchanged
 *   with each rank (the same in both directions).  A message to or from rank
 *   q carries these points ordered by the exchange index on the lower of the
 *   two ranks, so both sides agree.  FR_EMESH: a face or point without
 *   exactly one partner.  Host-only handles too (matching only).
 * fr_exchange_list: the boundary-point indices (fr_get_boundary_points
 *   order) of this part's exchanged points in message order; *n receives
 *   the count, points may be NULL.
 * fr_exchange_pack: gather, on the handle's stream, the traces of kind
 *   FR_XCH_SOLUTION (5 values per point: the stage input at the flux point)
 *   or FR_XCH_GRADIENT (after phase 1 of a Navier-Stokes stage: 15 gradient
 *   values per point with FP64 values, 5 viscous normal-flux values with
 *   FP32 / mixed values) into dev_buf [sum counts][nv] (value type: FP64 or
 *   FP32 as the mesh's values), messages in ascending rank order.
 * fr_exchange_unpack: the received buffer of the same layout into the
 *   partner-trace slots of the exchange points.
 * fr_rk_stage: one phase of stage `stage` of an RK step of `scheme`, on the
 *   handle's stream: phase 1, the NS common solution and gradients (nothing
 *   for Euler); phase 2, common fluxes, volume kernels and the stage's RK
 *   update (and the flux-point traces of the next stage).  part 1 launches
 *   only the work that needs no exchanged value (interior pairs, boundary
 *   points that are not exchange points, elements that own no exchange
 *   point), part 2 the rest, part 0 both: so the transport of a phase's
 *   input can overlap part 1.  Order per stage: pack/send/receive/unpack
 *   FR_XCH_SOLUTION (part 1 of phase 1 may run meanwhile), phase 1, then the
 *   same for FR_XCH_GRADIENT and phase 2 (Euler: only the solution exchange
 *   and phase 2).  Stage 0, phase 1, part 0 or 1 starts the step (dt); the
 *   last stage's phase 2 (part 0 or 2) synchronises the stream and returns
 *   FR_ENONFINITE / FR_ETIMEOUT from the device flag.  With
 *   FR_VARIANT_AUTO the part runs the default family (no tuning across
 *   processes).  FR_EINVAL: the entropy filter is on, or the mesh has
 *   exchange points and no fr_exchange_setup. */
enum { FR_XCH_SOLUTION = 0, FR_XCH_GRADIENT = 1 };
int fr_exchange_faces(const fr_mesh* mesh, int64_t* n_faces, int64_t* n_points,
                      int32_t* face_npts, double* centroids, double* pt_x,
                      double* pt_mag);
int fr_exchange_setup(fr_mesh* mesh, int rank, int nranks, const int64_t* faces_per_rank,
                      const int64_t* points_per_rank, const int32_t* face_npts,
                      const double* centroids, const double* pt_x,
                      const double* pt_mag, int64_t* counts);
int fr_exchange_list(const fr_mesh* mesh, int32_t* points, int64_t* n);
int fr_exchange_pack(fr_mesh* mesh, int what, void* dev_buf);
int fr_exchange_unpack(fr_mesh* mesh, int what, const void* dev_buf);
int fr_rk_stage(fr_mesh* mesh, int scheme, double dt, int stage, int phase, int part);

/* Viscous coupling of a Navier-Stokes mesh (the paper names the compressible
 * Navier-Stokes solver, not its interface scheme; reading of the local DG
 * flux).  Along every interface's orientation, whose "-" side is the
 * element with the lower global index (a boundary's inside is "-"), the
 * common solution is (1/2 - beta) u- + (1/2 + beta) u+, the viscous common
 * flux (1/2 + beta) F_v- + (1/2 - beta) F_v+, and the common normal flux
 * gains tau (u- - u+).  beta = tau = 0 (the default) is BR1; PyFR's LDG
 * default is beta = 1/2, tau = 0.1.  FR_EINVAL: not Navier-Stokes, beta
 * outside [-1/2, 1/2], tau negative or not finite, or beta != 0 on a member
 * of a partition group. */
int fr_set_viscous_scheme(fr_mesh* mesh, double beta, double tau);

/* Anti-aliasing (Section 3.2, "Anti-aliasing"): for qdeg > 0 the transformed
 * flux is no longer collocated at the solution points.  It is evaluated at
 * the points of a volume quadrature rule exact to degree qdeg (u and, for
 * Navier-Stokes, the corrected gradient interpolated there; the metric
 * evaluated there in the mesh's own form) and projected onto the solution
 * space by least squares, f~ = P f~_q; the divergence, correction and RK
 * update then use that f~.  Rules: n = qdeg/2 + 1 points per direction,
 * tensor Gauss-Legendre on hexahedra, collapsed Gauss-Legendre x
 * Gauss-Jacobi(1,0) [x Gauss-Jacobi(2,0)] on prisms and tetrahedra.
 * qdeg = 0 restores collocation.  qdeg in 0..24, else FR_EINVAL.  Adds per
 * element type the operators, the metric at the quadrature points ([ne][9]
 * [nq]) and a projected-flux buffer ([ne][15][nupts]) in device memory; the
 * vertex-metric and tensor-core volume kernels are not used while it is on.
 * Synchronises the handle's stream; later steps rebuild their graphs. */
int fr_set_antialias(fr_mesh* mesh, int qdeg);

/* Metric terms at the solution points: smat [n_elem][9][nupts] holds
 * S = det(J) J^{-1} (row-major 3x3 per point), rcpdjac [n_elem][nupts]
 * holds 1/det J.  Either pointer may be NULL. */
int fr_get_metrics(const fr_mesh* mesh, int etype, double* smat,
                   double* rcpdjac);

/* Number of interior flux-point pairs and boundary flux points. */
int fr_get_pairs(const fr_mesh* mesh, int64_t* n_interior,
                 int64_t* n_boundary);

/* Entropy filter (Section 3.2): when on, every RK stage of fr_rk_step
 * filters the new stage value of each element that violates rho >= 1e-8,
 * p >= 1e-8 or s = p rho^-gamma >= s_min (1 - 1e-8), s_min being the
 * minimum entropy of the stage input over the element's solution points,
 * its flux points and the partner flux points across its faces (1e-8 is
 * 2^-20 when the stage values are FP32: FR_FP32 and FR_MIXED).  The
 * filter multiplies modal coefficient k (orthonormal basis) by
 * exp(-zeta (d_k/p)^2), d_k the mode's total degree, with the smallest
 * zeta in [0, 36] that satisfies the constraints (bracketed Illinois
 * root-find, relative tolerance 1e-6, at most 24 margin evaluations;
 * constraints evaluated in FP64).  sample_capacity > 0 reserves a device
 * list of (4 features, zeta*) training samples, one per filtered element.
 * fr_rhs is never filtered. */
int fr_filter_enable(fr_mesh* mesh, int on, int64_t sample_capacity);

/* Learned start guess for the filter root-find: params holds the 1257
 * predictor parameters (W1[32][4], b1[32], W2[32][32], b2[32], W3[32], b3,
 * input mean[4], input std[4]); the library stores them in BF16 and
 * evaluates Linear(4,32)-SiLU-Linear(32,32)-SiLU-Linear(32,1)-softplus with
 * FP32 accumulation.  The guess only opens the root-find's bracket (at
 * z0, then z0 / r or r z0, then halving / doubling; r = params[1257] when
 * n = 1258, else 1.25); the exact root-find decides the result.  NULL
 * switches the predictor off. */
int fr_filter_set_mlp(fr_mesh* mesh, const float* params, int64_t n);

/* Filter the current solution in place, e.g. an initial state with
 * discontinuities; needs fr_filter_enable.  smin: host array of the
 * minimum-entropy bound of every element (element types in mesh order:
 * hex, prism, tet), or NULL to take it from the solution itself (then only
 * the positivity constraints can be active). */
int fr_filter_solution(fr_mesh* mesh, const double* smin);

/* Filter strength and margin evaluations of every element of `etype` in the
 * last filtered stage (zeta 0 and 1 evaluation for elements left alone). */
int fr_filter_last(const fr_mesh* mesh, int etype, float* zeta, int* evals);

/* Filter counters since the last reset: out[0] filtered element-stages,
 * out[1] margin evaluations in them, out[2] fallbacks (zeta = 36 still
 * infeasible), out[3] training samples written, out[4] element-stages that
 * used the predictor's guess. */
int fr_filter_stats(fr_mesh* mesh, uint64_t* out, int reset);

/* Copy up to `max` training samples ([n][5]: 4 features, zeta*) to host
 * memory and restart the sample list; *n receives the count. */
int fr_filter_samples(fr_mesh* mesh, float* out, int64_t max, int64_t* n);

/* Train the predictor on the GPU: full-batch Adam (learning rate lr) on the
 * mean squared error of log(predicted zeta) against log(zeta*), `epochs`
 * iterations, FP32, deterministic.  params (1257 floats) is the start and
 * receives the result; the 8 normalisation entries are not trained.
 * loss_hist (optional) receives the loss before each update. */
int fr_mlp_train(int device, const float* x, const float* zstar, int64_t n,
                 float* params, int epochs, float lr, float* loss_hist);

/* Loss and gradient of the same objective at params (grad: 1257 floats,
 * zeros for the normalisation entries). */
int fr_mlp_loss_grad(int device, const float* params, const float* x,
                     const float* zstar, int64_t n, float* loss, float* grad);

/* Measurement aid for the arithmetic roofline (the paper has no
 * counterpart): one launch of 8 x (number of SMs) blocks of 256 threads,
 * each thread running eight independent chains of `iters` fused
 * multiply-adds in FR_DTYPE_F64 or FR_DTYPE_F32, after one shorter warm-up
 * launch.  *ms: device time of the timed launch (CUDA events), *flops:
 * 2 * 8 * iters * threads.  Allocates and frees a small output buffer on
 * `device`; synchronous. */
int fr_probe_fma(int device, int dtype, int64_t iters, double* ms, double* flops);

/* Self-check of the arithmetic the library does off the FP64 pipe (the
 * paper has no counterpart): the mixed form widens FP32 increments to FP64
 * and rounds its FP64 registers to FP32 with integer instructions, and the
 * entropy filter's FP64 checks take 1/rho and fifth roots by Newton steps
 * from FP32 values.  Runs n seeded patterns (random bits, exponents around the
 * FP32 range, exact rounding ties, carries into and out of the exponent) on
 * `device` and writes to *mismatches the number of conversions that differ
 * from the hardware conversions in any bit (NaNs: that differ in NaN-ness)
 * plus the reciprocals more than 2 units in the last place from the FP64
 * division and the fifth roots r with |r^5 - x| > 5e-15 x.
 * Allocates and frees 8 bytes on `device`; synchronous. */
int fr_check_conversions(int device, uint64_t seed, int64_t n, int64_t* mismatches);

/* Message of the last failed call on this thread. */
const char* fr_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FRGB_H */
