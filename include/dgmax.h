/*
 * dgmax.h -- C ABI of the GB300 matrix-free discontinuous Galerkin
 * time-domain Maxwell solver (Kapidani & Schoeberl, arXiv 2002.08733).
 *
 * Problem statement (Sec. I, Eqs. (ampere_cont)/(faraday_cont)): on a
 * tetrahedral mesh of a domain with per-element permittivity eps and
 * permeability mu, advance the electric and magnetic fields from initial
 * values, with PEC walls on the boundary (Sec. IV) and an optional Cartesian
 * PML (Sec. IV, complex stretching) around a box, driven by point dipoles.
 *
 * Discretisation (Secs. II-III): per element, every field component is
 * expanded in the orthonormal modal basis of degree p on the reference
 * tetrahedron (Eq. (dubiner_functions), standard collapsed exponents; modes
 * graded by total degree, then i, then j), mapped covariantly
 * (Eq. (mapped_eh)).  The state of one column is, per element, 3 covariant
 * coefficient vectors of E and 3 of H with N = (p+1)(p+2)(p+3)/6 modes each.
 * The element map uses the element's vertices in ascending global id order.
 *
 * Memory layout of a field buffer ("fields"): real numbers (double for
 * DGM_FP64, float for DGM_FP32), index ((c * N + l) * K + e) * S + s for
 * component c in 0..5 (Ex, Ey, Ez, Hx, Hy, Hz), mode l, element e, column s.
 * Auxiliary PML buffers ("aux") use the same layout with K replaced by the
 * number of PML elements (dgm_info.n_pml) in ascending element order;
 * components 0..2 hold p, 3..5 hold q (Eqs. (p_variable), (q_variable)).
 *
 * Ownership: host inputs are copied by dgm_plan_create.  All device memory
 * belongs to the caller and is passed by pointer to dgm_bind; the library
 * allocates no device memory.  Calls are asynchronous on the bound stream
 * unless stated otherwise.
 *
 * Errors: every call returns DGM_OK or one of the codes below; the message
 * of the last error of the calling thread is returned by dgm_last_error().
 * Device-side errors are latched in a status word inside the geometry buffer
 * and reported by the next synchronising call (dgm_energy, dgm_status_check).
 */
#ifndef DGMAX_H
#define DGMAX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DGM_OK 0
#define DGM_EINVAL 1   /* invalid argument */
#define DGM_EMESH 2    /* degenerate element, non-manifold face, bad vertex id */
#define DGM_EUNSUP 3   /* unsupported order / precision / combination */
#define DGM_ECUDA 4    /* CUDA runtime error */
#define DGM_ETIMEOUT 5 /* a device-side wait gave up */
#define DGM_ENAN 6     /* non-finite values detected */
#define DGM_ESTATE 7   /* call out of order (e.g. not bound) */

#define DGM_FP64 0
#define DGM_FP32 1

#define DGM_CENTRAL 0  /* central flux, Eqs. (uwc)/(cwc) */
#define DGM_UPWIND 1   /* upwind (Riemann) flux */

#define DGM_LEAPFROG 0 /* staggered leapfrog, Sec. V (central flux only) */
#define DGM_LSRK4 1    /* five-stage low-storage RK4 (Carpenter & Kennedy) */

typedef struct dgm_plan dgm_plan;

typedef struct {
    int32_t p;          /* polynomial degree of E and H, 1..4 (FP64) or 1..5 (FP32) */
    int32_t precision;  /* DGM_FP64 or DGM_FP32 field arithmetic; geometry is FP64 */
    int32_t flux;       /* DGM_CENTRAL or DGM_UPWIND */
    int32_t integrator; /* DGM_LEAPFROG or DGM_LSRK4 */
    int32_t n_columns;  /* S >= 1 independent problems (sources) sharing the mesh */
    int32_t max_receivers; /* capacity for dgm_set_receivers (0: none) */
    double dt;          /* time step */
} dgm_options;

/* Cartesian PML (Sec. IV): the layer is everything outside the box [lo, hi].
 * Per element the damping triple is sigma_a = sigma_max (d_a / thickness)^order
 * at the element centroid, d_a its depth into the layer along axis a; the
 * element then carries eta, xi tensors and auxiliary fields p, q. */
typedef struct {
    double lo[3];
    double hi[3];
    double thickness;
    double sigma_max;
    int32_t order;
    int32_t reserved;
} dgm_pml;

typedef struct {
    int64_t K;            /* elements */
    int64_t n_pml;        /* elements carrying auxiliary fields */
    int32_t N;            /* modes per component */
    int32_t NF;           /* modes per face component */
    int32_t S;            /* columns */
    int32_t real_size;    /* bytes per real of the field buffers (4 or 8) */
    size_t bytes_fields;  /* one field buffer: 6 N K S reals */
    size_t bytes_aux;     /* one auxiliary buffer: 6 N n_pml S reals (0 without PML) */
    size_t bytes_geom;    /* geometry + workspace buffer, 256-byte aligned start */
    int32_t n_quad;       /* projection quadrature points per element */
    int32_t N_H;          /* modes per H component: N, except on a mixed-order plan */
    int64_t n_facets;     /* interior facets carrying the penalty's facet field (0: off) */
    size_t bytes_facets;  /* one facet-field buffer: n_facets * S * 3 * NF reals */
} dgm_info;

/* Create a plan: validates the mesh, sorts each element's vertices, builds the
 * face-neighbour table, geometric factors (A^-T, det A), PML tensors and the
 * reference curl/trace matrices (Sec. III, Eq. (matrix_free_curl)).
 * xyz: [nv][3] vertex coordinates; tets: [nt][4] vertex ids (any order);
 * eps, mu: [nt] positive per-element material values; pml may be NULL.
 * Errors: DGM_EINVAL, DGM_EMESH, DGM_EUNSUP.  No CUDA call is made. */
int dgm_plan_create(dgm_plan** out, int64_t nv, const double* xyz, int64_t nt,
                    const int64_t* tets, const double* eps, const double* mu,
                    const dgm_pml* pml, const dgm_options* opt);

/* Mixed orders (Sec. III, Eqs. (triale)/(trialh)): E of degree opt->p + 1 and
 * H of degree opt->p, as the paper discretises them.  Every operator is a
 * submatrix of the degree-(p+1) reference operators (hierarchical orthonormal
 * bases; checked at creation).  Field buffers hold E component c, mode l at row
 * c N + l (N = dgm_info.N, E's modes) and H component c, mode l at row
 * 3 N + c N_H + l; bytes_fields covers 3 (N + N_H) rows.  Supports LSRK4 (and
 * dgm_rhs) with central or upwind flux, FP64 and FP32, p = 1..3, sources,
 * receivers, projection, energy and partitions; no PML, leapfrog, adjoint or
 * batch (DGM_EUNSUP / DGM_EINVAL).  Runs a plain one-thread-per-column kernel
 * with dense operators.  Otherwise as dgm_plan_create. */
int dgm_plan_create_mixed(dgm_plan** out, int64_t nv, const double* xyz, int64_t nt,
                          const int64_t* tets, const double* eps, const double* mu,
                          const dgm_pml* pml, const dgm_options* opt);

/* Sizes and counts of a plan.  No CUDA call. */
int dgm_plan_info(const dgm_plan* plan, dgm_info* out);

/* Bind caller-owned device buffers and a CUDA stream (cudaStream_t, may be 0)
 * and upload the geometry asynchronously.  geom: bytes_geom bytes, 256-byte
 * aligned; fields0/fields1/res: bytes_fields each (fields1 and res may be NULL
 * for leapfrog); aux0/aux1/aux_res: bytes_aux each (NULL without PML).
 * The state lives in fields0 at bind time; see dgm_current. */
int dgm_bind(dgm_plan* plan, void* geom, void* fields0, void* fields1, void* res,
             void* aux0, void* aux1, void* aux_res, void* stream);

/* Point dipoles, one per listed column: j = dir delta(r - pos) g(t),
 * g(t) = sin(2 pi f0 (t - t0)) exp(-(t - t0)^2 / (2 s^2)), s = 1/(2 pi bw).
 * Enters the E equation as -(j, phi)_T in the element containing pos.
 * Arrays have n entries (pos, dir: 3 each).  Requires a bound plan; uploads
 * asynchronously.  Errors: DGM_EINVAL (point outside the mesh, bad column). */
int dgm_set_sources(dgm_plan* plan, int32_t n, const int32_t* column, const double* pos,
                    const double* dir, const double* f0, const double* bw, const double* t0);

/* Receivers: points at which dgm_sample_receivers evaluates E.  n <= the
 * plan's max_receivers; pos: host [n][3].  Each point is located in the
 * lowest-index element containing it.  Requires a bound plan (uploads and
 * synchronises).  Errors: DGM_EINVAL (too many, or a point outside the mesh). */
int dgm_set_receivers(dgm_plan* plan, int32_t n, const double* pos);

/* Physical E at the receivers for every column, E(r) = A^-T sum_l u_l phi_l(r_hat)
 * (Eq. (mapped_eh)): out_device[s][r][3] doubles (device), computed from the
 * device field buffer `fields` on the bound stream (asynchronous). */
int dgm_sample_receivers(dgm_plan* plan, const void* fields, double* out_device);

/* One evaluation of the semi-discrete right-hand side at time t (the hot
 * path of one stage: reference-curl volume term, face traces, numerical flux,
 * lift, 3x3 mass-block inverse, PML terms, sources):
 * dfields = d(fields)/dt, daux = d(aux)/dt (aux/daux NULL without PML).
 * All pointers are device buffers in the layout above. */
int dgm_rhs(dgm_plan* plan, const void* fields, const void* aux, void* dfields, void* daux,
            double t);

/* Leapfrog only: the half step H <- H + dt/2 L_H(E) that starts the staggered
 * scheme from H given at time t0 (Sec. V). */
int dgm_leapfrog_start(dgm_plan* plan, double t0);

/* Advance the bound state n_steps time steps from time t0 (asynchronous).
 * LSRK4 ping-pongs between fields0 and fields1 (and aux0/aux1). */
int dgm_advance(dgm_plan* plan, int64_t n_steps, double t0);

/* Batched advance of several independent problems (the batching pattern of
 * many sources and uneven problems): a batch groups bound LSRK4 plans of any
 * order/precision; dgm_batch_advance advances every member by n_steps using
 * one CUDA graph launch per two time steps, inside which the members' stage
 * kernels run concurrently on forked streams (each member keeps its own time
 * step, sources and buffers).  The graph is captured at creation.  Member
 * times live in device memory (a slot of each member's geometry buffer), so
 * sources see the right time in every replay.  Ordering: the batch waits for
 * work already queued on the members' bound streams and the members' streams
 * wait for the batch.  stream: the caller's stream (cudaStream_t, may be 0),
 * ordered before and after each advance; the graph itself runs on a stream
 * the batch owns.  Errors: DGM_EINVAL (no members, unbound or non-LSRK4 member,
 * duplicate member), DGM_ECUDA. */
typedef struct dgm_batch dgm_batch;
int dgm_batch_create(dgm_batch** out, dgm_plan* const* members, int32_t n, void* stream);
/* t0: host array of n start times (NULL: all 0).  Asynchronous. */
int dgm_batch_advance(dgm_batch* batch, int64_t n_steps, const double* t0);
void dgm_batch_destroy(dgm_batch* batch);

/* Replace the per-element materials of a plan (host arrays [K]); uploads if
 * bound (synchronous).  The geometry and everything else are kept. */
int dgm_set_materials(dgm_plan* plan, const double* eps, const double* mu);

/* Discrete adjoint of LSRK4 time stepping with receivers (gradient of a loss
 * of the receiver records with respect to per-element eps and mu).
 *
 * dgm_forward_record advances the bound state n_steps from time t0 (like
 * dgm_advance), writes the receiver records after every step to
 * records_device [n_steps][S][R][3] (doubles, R = receivers set) and keeps a
 * checkpoint every seg = ceil(sqrt(n_steps / 5)) steps in `workspace`.
 * dgm_adjoint then runs the adjoint backwards in time from dL/drecords
 * (device, same layout as the records): each checkpoint segment is
 * recomputed forward once, keeping the five stage inputs of each of its
 * steps (n_steps / seg + 5 seg states in all), and the transposed stage
 * kernels accumulate the gradient per column in FP64; deps_device and
 * dmu_device (doubles [K]) receive dL/d eps_T and dL/d mu_T summed over
 * columns.  workspace: device memory of dgm_adjoint_workspace bytes,
 * 256-byte aligned, owned by the caller, shared by the two calls.  The
 * adjoint stage matches the discrete transpose of the forward stage exactly
 * (same reference operators, flux, PML, sources). */
int dgm_adjoint_workspace(const dgm_plan* plan, int64_t n_steps, size_t* bytes);
int dgm_forward_record(dgm_plan* plan, int64_t n_steps, double t0, double* records_device,
                       void* workspace);
int dgm_adjoint(dgm_plan* plan, int64_t n_steps, double t0, const double* drecords_device,
                void* workspace, double* deps_device, double* dmu_device);

/* Autotuner: times each compiled tile shape (columns per CTA x threads per
 * CTA) of the LSRK4 stage kernel on the plan's current state, `reps` launches
 * each, and keeps the fastest for later dgm_advance / dgm_batch_create calls;
 * then times the tile visiting orders of dgm_set_tile_groups for that shape
 * (at least ten launches each) and, where the plan has the phase-1 bulk copies
 * of dgm_set_tile_loads, those against per-thread loads (each twice, the
 * faster of its two times), keeping per-thread loads only when they are
 * faster.  The plan's state is only read.  An LSRK4
 * plan is timed on stage sequences as dgm_advance runs them: the first launch
 * reads the state and writes `workspace`, later ones alternate between
 * `workspace` and the plan's second field (and auxiliary) buffer, which hold
 * nothing between steps; other plans write `workspace` only.  workspace:
 * device memory of 2*align256(bytes_fields) + 2*align256(bytes_aux) bytes,
 * 256-byte aligned.  ms_out (host, may be NULL) receives the mean time per
 * launch of each variant.  Synchronises the bound stream. */
int dgm_autotune(dgm_plan* plan, void* workspace, int32_t reps, float* ms_out);
int dgm_autotune_info(const dgm_plan* plan, int32_t* n_variants, int32_t* chosen);
/* Select a tile-shape variant explicitly (0 .. n_variants-1). */
int dgm_set_variant(dgm_plan* plan, int32_t variant);
/* Index arithmetic of the stage kernels.  By default (force = 0) a launch
 * uses 32-bit indices when every index it forms fits (field and face-jump
 * rows times columns, auxiliaries, geometry, the per-face table are all below
 * 2^32) and 64-bit indices otherwise; force = 1 selects the 64-bit kernels
 * always, to check that path on problems of any size.  Results are the same
 * either way.  DGM_EINVAL for other values. */
int dgm_set_index64(dgm_plan* plan, int32_t force);
/* How the single-column stage kernels bring a tile's coefficients, element
 * constants and face constants into shared memory.  Where the plan allows it
 * (one column per element, S = 1; rows of the field and table buffers on
 * 16-byte boundaries, i.e. K a multiple of 4 in FP32 and of 2 in FP64; the
 * stage reads one of the two bound field buffers) dgm_bind builds tensor maps
 * and phase 1 moves the tile with a few tiled bulk copies (TMA) issued by one
 * thread; otherwise every thread loads and stores its share of rows.
 * per_thread = 1 forces the per-thread loads, 0 (the default) restores the
 * automatic choice; the results are the same bits either way.  DGM_EINVAL for
 * other values.  dgm_get_tile_loads sets *bulk to 1 when the next stages of a
 * bound plan use the bulk copies, else 0.  A bulk copy that has not completed
 * within 0.5 s leaves its tile unwritten and latches DGM_ETIMEOUT in the
 * device status word (dgm_status_check). */
int dgm_set_tile_loads(dgm_plan* plan, int32_t per_thread);
int dgm_get_tile_loads(const dgm_plan* plan, int32_t* bulk);
/* Order in which the stage and adjoint kernels visit their column tiles:
 * with groups = G > 1 (and a tile count that G divides) consecutive CTAs
 * take tiles from G equal segments of the columns in turn, which keeps the
 * neighbours' coefficients of meshes numbered in G blocks (e.g. a Kuhn grid
 * numbered by tetrahedron type) in L2; 1 = plain order.  Results do not
 * depend on it.  dgm_autotune picks it after the tile shape: the fastest of
 * 1, 2, 3, 4, 6, 8, 12, or 1 unless that is at least 1 % faster than the plain
 * order; DGM_EINVAL outside 1..64. */
int dgm_set_tile_groups(dgm_plan* plan, int32_t groups);
int dgm_get_tile_groups(const dgm_plan* plan, int32_t* groups);

/* Index (0 or 1) of the bound field/aux buffer that holds the current state. */
int dgm_current(const dgm_plan* plan);

/* Same as dgm_advance but end to end from host memory: copies fields_in
 * (host, bytes_fields) to the current device buffer, advances, copies the
 * result back to fields_out (host) and synchronises the stream. */
int dgm_advance_host(dgm_plan* plan, const void* fields_in, void* fields_out,
                     int64_t n_steps, double t0);

/* Discrete energy 1/2 (e . M_eps e + h . M_mu h) per column, accumulated in
 * FP64 (Sec. III, energy conservation of the central flux).  out: host [S].
 * Synchronises the stream.  A non-finite energy (a NaN or an overflow in the
 * column's state) latches DGM_ENAN in the device status word and the call
 * returns DGM_ENAN (out still holds the energies). */
int dgm_energy(dgm_plan* plan, const void* fields, double* out);

/* Element ids of the PML elements in auxiliary-buffer order (ascending):
 * host out[n_pml].  No CUDA call. */
int dgm_pml_elements(const dgm_plan* plan, int64_t* out);

/* Physical quadrature points used by dgm_project: host [K][n_quad][3]. */
int dgm_quad_points(const dgm_plan* plan, double* xyz_out);

/* L2 projection of initial values onto the covariant basis (Sec. II).
 * samples: host [K][n_quad][6] values of (Ex, Ey, Ez, Hx, Hy, Hz) at the
 * points of dgm_quad_points; writes column `column` of the device buffer
 * `fields` (synchronous copy on the bound stream). */
int dgm_project(dgm_plan* plan, const double* samples, int32_t column, void* fields);

/* Energy per column, like dgm_energy, but for callers that must not allocate.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot let the library touch the device allocator, e.g. a latency-critical
 * stepping loop in which a cudaMalloc/cudaFree would synchronise the device,
 * or a host application whose device memory is owned entirely by another
 * framework's allocator.  It allocates nothing and makes no allocating call;
 * its reduction scratch is a fixed array inside the library (file-scope
 * device memory, DGM_NOALLOC_MAX_COLUMNS * 304 doubles = 152 KiB, held by
 * every GPU that loads the library until the process exits).
 *
 * fields: device field buffer of the plan; out_device: device array of S
 * doubles receiving the energies (written on the bound stream, no host
 * synchronisation).  Errors: DGM_EINVAL if the plan has more than
 * DGM_NOALLOC_MAX_COLUMNS columns, DGM_ESTATE if not bound.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one scratch array (each
 * call overwrites every entry it later reads, so nothing needs clearing):
 * calls whose kernels overlap on the GPU (other streams, other threads)
 * race and must be ordered by the caller. */
#define DGM_NOALLOC_MAX_COLUMNS 64
int dgm_energy_noalloc(dgm_plan* plan, const void* fields, double* out_device);

/* ---- One mesh on several GPUs: element partitions with a halo exchange ----
 *
 * The right-hand side of an element (Secs. III-IV: volume curl, face traces,
 * numerical flux, lift, mass inverse) reads only its own coefficients and
 * those of its face neighbours.  A part of the mesh therefore advances on its
 * own GPU if, before every stage, it holds current copies of the
 * coefficients of the other parts' elements that share a face with it (its
 * halo).  The library partitions, builds the halo lists, packs and unpacks
 * halo coefficients and runs single stages; moving the packed buffers between
 * GPUs (NCCL send/receive, or a copy into the receiver's own memory) is the
 * caller's. */

/* Slab partition: elements sorted by centroid coordinate along `axis` (0, 1,
 * 2; ties by element id) and cut into nparts contiguous runs of nearly equal
 * size (k-plane slabs on a Kuhn grid).  part: host [nt] part ids.  No CUDA
 * call.  Errors: DGM_EINVAL, DGM_EMESH. */
int dgm_partition_slabs(int64_t nv, const double* xyz, int64_t nt, const int64_t* tets,
                        int32_t axis, int32_t nparts, int32_t* part);

typedef struct {
    int64_t n_owned;   /* elements of this part */
    int64_t n_ghost;   /* other parts' elements that share a face with this part */
    int64_t n_send;    /* total entries of send_idx (an element may go to two peers) */
    int64_t n_recv;    /* total entries of recv_idx (= n_ghost) */
    int32_t n_peers;   /* parts this part exchanges with */
    int32_t reserved;
} dgm_halo_sizes;

/* Local numbering and halo lists of part `rank` of a partition (part[nt]):
 * local element i < n_owned is the i-th owned element in ascending global
 * id, local element n_owned + j the j-th ghost in ascending global id
 * (local_to_global: [n_owned + n_ghost]).  Per peer q (peers[n_peers],
 * ascending): send_idx holds send_count[q] local ids of owned elements whose
 * coefficients peer q needs, recv_idx recv_count[q] local ids of the ghosts
 * peer q owns, both in ascending global id, so that a part's send list to q
 * and q's receive list from it match entry by entry; lists are stored peer
 * after peer.  With local_to_global NULL only *sizes is filled.  All arrays
 * are host memory, caller-owned.  No CUDA call. */
int dgm_halo_build(int64_t nt, const int64_t* tets, const int32_t* part, int32_t nparts,
                   int32_t rank, dgm_halo_sizes* sizes, int64_t* local_to_global,
                   int32_t* peers, int64_t* send_count, int64_t* send_idx,
                   int64_t* recv_count, int64_t* recv_idx);

/* Only the first n elements of the plan are updated by the stage kernels
 * (dgm_rhs, dgm_stage, dgm_advance, dgm_autotune) and summed by dgm_energy;
 * the others are halo copies that the caller keeps current.  1 <= n <= K
 * (default K).  Plans with fewer active elements reject the adjoint and
 * the batch.  No CUDA call. */
int dgm_set_active(dgm_plan* plan, int64_t n);

/* Gather the coefficients of n elements (local ids idx_device[n], int64,
 * device) of the field buffer `fields` into buf_device [6N][n][S] (real
 * numbers of the plan's precision, device), or scatter them back
 * (unpack).  Asynchronous on the bound stream. */
int dgm_halo_pack(dgm_plan* plan, const void* fields, const int64_t* idx_device, int64_t n,
                  void* buf_device);
int dgm_halo_unpack(dgm_plan* plan, void* fields, const int64_t* idx_device, int64_t n,
                    const void* buf_device);

/* One stage k (0..4) of the LSRK4 step that starts at time t: reads the
 * current field (and auxiliary) buffer, writes the other one and the
 * residuals, and makes it current (dgm_current).  Five calls with k = 0..4
 * equal dgm_advance(plan, 1, t); between them a partitioned run refreshes
 * the halo of the new current buffer.  Asynchronous. */
int dgm_stage(dgm_plan* plan, int32_t k, double t);

/* Incident plane wave (Sec. V, the PEC-sphere scattering set-up: a plane
 * wave in a given direction with a smooth time envelope; Appendix A, the
 * incidentfield boundary): E_inc(r, t) = E0 g(t - t0 - d . r / speed),
 * g(x) = cos(2 pi f0 x) exp(-x^2 / (2 s^2)), s = 1 / (2 pi bw); f0 = 0 and
 * s = w / sqrt(2) give the paper's exp(-((t - t0) / w)^2).  direction is used
 * as given (pass a unit vector). */
typedef struct {
    double E0[3];         /* polarisation and amplitude */
    double direction[3];  /* propagation direction d */
    double speed;         /* phase speed (> 0) */
    double f0, bw, t0;    /* carrier frequency, bandwidth (> 0), delay */
} dgm_incident;

/* Make n boundary faces (faces[n][3]: vertex ids, any order; host memory)
 * incident faces: there the exterior state is e+ = e- + 2 E_inc, h+ = -h-
 * with the element's own impedance (a magnetic wall that radiates the
 * incident field into the mesh; the upwind flux absorbs what arrives from
 * inside).  All columns see the same wave.  n = 0 restores PEC on every
 * boundary face.  A later call replaces the previous set.  On a bound plan
 * uploads the table and the neighbour codes (synchronises the stream).  The
 * stage launches then evaluate the wave's face-mode integrals at each stage
 * time (collapsed Gauss rule with (p + 6)^2 points per face, FP64).
 * Errors: DGM_EINVAL (a face that is not a boundary face, given twice, bad
 * wave parameters); DGM_EUNSUP on mixed-order and leapfrog plans.  A plan
 * on a paired FP32 stage variant moves to variant 0; afterwards the paired
 * variants are refused (dgm_set_variant) or skipped (dgm_autotune), and
 * the adjoint and the batch refuse the plan. */
int dgm_set_incident(dgm_plan* plan, int64_t n, const int64_t* faces, const dgm_incident* wave);

/* Symmetric interior penalty with a facet field (Sec. III, Eqs. (jmp_var_def),
 * (1st_weak_equation), (weak_penalty), in the skew matrix form printed after
 * them): every interior facet F carries a tangential field h_s of degree p,
 *   E equation of both sides:  (eps de/dt, phi)_T += -(h_s x n_T, phi)_F
 *   facet field:  (mu_F / alpha) (dh_s/dt, psi)_F = (n- x (e- - e+), psi)_F
 * with T- the side of lower element index (its outward normal n-) and mu_F
 * the mean of both sides' mu; alpha > 0 (0 turns the penalty off).  Call
 * before dgm_bind.  Central flux and LSRK4 only, no PML, no mixed orders
 * (DGM_EUNSUP).  Facets are numbered by (lower element, its local face),
 * ascending; dgm_info gives their count and the facet buffer size.  The
 * paired FP32 variants are then refused or skipped, like the adjoint and the
 * batch.  No CUDA call. */
int dgm_set_sip(dgm_plan* plan, double alpha);

/* Caller-owned device buffers of the facet field (dgm_info.bytes_facets each;
 * layout [3][NF][facet][column]: physical Cartesian components of h_s per
 * face mode of the facet's face basis): hs0 holds the current facet state
 * (zero for a start from rest) and alternates with hs1 like the field
 * buffers; hs_res is the LSRK residual, and dgm_rhs writes dh_s/dt of the
 * current facet state into it.  Call after dgm_bind.  dgm_energy does not
 * include the facet energy. */
int dgm_bind_sip(dgm_plan* plan, void* hs0, void* hs1, void* hs_res);

/* Read and clear the device status word (synchronises).  Returns DGM_OK or
 * the latched device error. */
int dgm_status_check(dgm_plan* plan);

/* Message of the calling thread's last error ("" if none). */
const char* dgm_last_error(void);

void dgm_plan_destroy(dgm_plan* plan);

#ifdef __cplusplus
}
#endif

#endif /* DGMAX_H */
