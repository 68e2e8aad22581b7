/*
 * nsi_assemble.h -- C ABI of the GB300 (sm_103a) incompressible-flow P1
 * tetrahedral matrix assembly library (libnsi_assemble.so).
 *
 * The operation is the element matrix assembly of Alya's incompressible
 * Navier-Stokes module (paper Section II-A, Listings 1 and 2): for every
 * linear tetrahedron (4 nodes, 3 dimensions) gather nodal coordinates and
 * velocities through the connectivity (calculate_transients), form the
 * Jacobian, its determinant and inverse and the Cartesian shape-function
 * gradients (calculate_cartesian_derivatives), integrate the convection,
 * viscous and pressure-gradient terms at 4 Gauss points (Table I rows
 * calculate_gauss_point_values ... calculate_viscous_term) and scatter-add
 * the element matrices and right-hand side into global arrays
 * (perform_assembly_in_global_system).  The per-term formulas are the
 * Galerkin P1 form, because the paper names the subroutines but does not
 * print their equations:
 *
 *   A_e[a][b]    = int rho N_a (u_h . grad N_b) + mu grad N_a . grad N_b
 *                  + delta_ab rho |T_e| / (4 dt)            (4x4, scalar per node)
 *   G_e[a][b][d] = - int d_d N_a N_b                        (4x4x3)
 *   b_e[a][k]    = rho (|T_e| / 4) u^n_{a,k} / dt           (4x3, lumped)
 *
 * and A = sum_e A_e, G = sum_e G_e on one CSR pattern, rhs = sum_e b_e.
 *
 * Conventions shared by every entry point:
 *  - All array pointers in NsiMesh, NsiFields and NsiOutputs are DEVICE
 *    pointers unless the entry point says otherwise.  The caller owns every
 *    input and output buffer and every stream; a handle owns only what it
 *    builds at create time (CSR pattern, element colouring, gather maps,
 *    packed coordinates) plus a device error word.
 *  - Node arrays are structure-of-arrays, length n_nodes.  Connectivity is
 *    int32 [n_elems][4], 0-based (Alya's lnods is 1-based Fortran; callers
 *    subtract 1).  Every element must be positively oriented (det J > 0).
 *  - CSR: row_ptr int32 [n_nodes + 1], col_idx int32 [nnz], columns strictly
 *    ascending within a row: every node pair sharing an element (so the
 *    diagonal of every node that belongs to an element; a node in no element
 *    has an empty row and a zero right-hand side).  A_val is [nnz]; G_val is
 *    component-major [3][nnz]; rhs is component-major [3][n_nodes].
 *  - Precision (fixed per handle):
 *      NSI_FP64            u, u_n: double;  A, G, rhs: double.  All element
 *                          arithmetic and accumulation in IEEE double.
 *      NSI_MIXED_F32_ACC64 u, u_n: float;   A, G, rhs: double.  Gathers and
 *                          element arithmetic in float (coordinates kept as
 *                          float hi/lo pairs so edge vectors keep ~48 bits);
 *                          A's off-diagonal entries and G summed in float
 *                          (each the few element terms of one edge, float
 *                          products: about 1e-7 of the row's largest entry);
 *                          A's diagonal (the lumped mass minus its row's
 *                          other entries, where the row's terms cancel), the
 *                          lumped mass and the RHS as compensated float
 *                          pairs (about 48 significant bits); stored as
 *                          double.  The element-centric modes (colour,
 *                          atomic) add in double.
 *      NSI_MIXED_F32_ACC32 u, u_n: float;   A, G, rhs: float.
 *  - Outputs are OVERWRITTEN by every assemble call (the call defines every
 *    entry; no prior zeroing is needed).
 *  - The device entry points (nsi_assemble, _mode, _batched, _convective,
 *    _nodal, _stabilized, _vjp, nsi_residual) never allocate device memory, never
 *    synchronise the stream, and only enqueue work on the given stream; they
 *    may be captured into a CUDA graph.  nsi_assemble_host, for host buffers,
 *    is the exception (see its comment).  Errors detected on the device (only when the handle
 *    was created with debug_checks) are reported by nsi_device_status().
 *  - Every function returns an nsi_status; on failure nsi_last_error()
 *    returns a human-readable message for the calling thread.  No C++
 *    exception crosses this ABI.
 */
#ifndef NSI_ASSEMBLE_H
#define NSI_ASSEMBLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NSI_ABI_VERSION 2

typedef struct NsiHandle NsiHandle; /* opaque; one per mesh */

typedef enum {
    NSI_OK = 0,
    NSI_ERR_INVALID_ARG = 1,   /* NULL pointer, negative size, bad enum, bad dt */
    NSI_ERR_BAD_MESH = 2,      /* node index out of range or det J <= 0 */
    NSI_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    NSI_ERR_OOM = 4,           /* device or host allocation failed */
    NSI_ERR_UNSUPPORTED = 5,   /* option not available for this mesh/precision */
    NSI_ERR_TIMEOUT = 6,       /* a bounded device wait gave up */
    NSI_ERR_DEVICE_CHECK = 7   /* a device-side bounds check fired */
} nsi_status;

typedef enum {
    NSI_FP64 = 0,
    NSI_MIXED_F32_ACC64 = 1,
    NSI_MIXED_F32_ACC32 = 2
} nsi_precision;

typedef enum {
    NSI_SCATTER_AUTO = 0,     /* library choice (row gather when available) */
    NSI_SCATTER_COLOR = 1,    /* element colouring, plain read-add-write, deterministic */
    NSI_SCATTER_ATOMIC = 2,   /* one element per thread, global atomic adds */
    NSI_SCATTER_GATHER = 3    /* one CSR row per thread, gathers its elements, writes once;
                                 deterministic (rows of more than 32 entries by a second,
                                 per-row kernel: NsiInfo.long_rows) */
} nsi_scatter;

typedef struct {
    int64_t n_nodes;
    int64_t n_elems;
    const int32_t* lnods; /* device int32 [n_elems][4], 0-based */
    const double* x;      /* device double [n_nodes] */
    const double* y;
    const double* z;
} NsiMesh;

typedef struct {
    int32_t precision;    /* nsi_precision */
    int32_t scatter;      /* nsi_scatter: default mode of nsi_assemble for this handle */
    int32_t block;        /* threads per block, 0 = library default */
    int32_t debug_checks; /* 1: kernels bounds-check every index they load */
    int32_t reserved[4];  /* must be 0 */
} NsiOptions;

typedef struct {
    const void* u[3];   /* device velocity components [n_nodes], double or float by precision */
    const void* u_n[3]; /* velocity entering the RHS; NULL entries mean "same as u" */
    double rho;         /* density */
    double mu;          /* dynamic viscosity */
    double dt;          /* time step, > 0 */
} NsiFields;

typedef struct {
    void* A_val; /* device [nnz], double or float by precision (may be NULL when nnz = 0) */
    void* G_val; /* device [3][nnz] (may be NULL when nnz = 0) */
    void* rhs;   /* device [3][n_nodes] */
} NsiOutputs;

/*
 * Build a handle for one mesh: validates the connectivity (indices in range,
 * every det J > 0, computed in double on the host), builds the CSR pattern of
 * all node pairs sharing an element, the row-gather maps, a greedy element
 * colouring and packed coordinate copies.  Synchronous; allocates device
 * memory owned by the handle.  `stream` (a cudaStream_t, may be NULL) is used
 * for the uploads.  On failure *out is NULL.
 * Paper: the CSR pattern is where perform_assembly_in_global_system (Listing
 * 2, Section II-A) adds the element matrices; the paper's kernel receives the
 * mesh once and assembles every time step (Section II), so the pattern and
 * the gather maps are built once per mesh here.
 */
nsi_status nsi_assemble_create(const NsiMesh* mesh, const NsiOptions* opts, void* stream,
                               NsiHandle** out);

/* Release a handle (NULL is allowed).  Synchronises the device first.
 * (No counterpart in the paper: resource management of this library.) */
nsi_status nsi_assemble_destroy(NsiHandle* h);

/*
 * The handle's CSR pattern (device pointers owned by the handle, valid until
 * destroy) and its sizes.  Any output pointer may be NULL.
 * (No counterpart in the paper: the pattern of the global matrix of
 * Section II-A, exposed to the caller.)
 */
nsi_status nsi_csr_pattern(const NsiHandle* h, const int32_t** row_ptr, const int32_t** col_idx,
                           int64_t* nnz);

/*
 * Copy the handle's CSR pattern into caller buffers (host or device;
 * row_ptr: n_nodes + 1 entries, col_idx: nnz entries; either may be NULL).
 * Enqueued on `stream`, which is then synchronised.  (No counterpart in the
 * paper; as nsi_csr_pattern.)
 */
nsi_status nsi_csr_pattern_copy(const NsiHandle* h, int32_t* row_ptr, int32_t* col_idx, void* stream);

/* Sizes and facts about the handle: nodes, elements, nnz, colours, max row
 * length, launch choices.  (No counterpart in the paper.) */
typedef struct {
    int64_t n_nodes, n_elems, nnz;
    int32_t n_colors, max_row, precision, scatter;
    int64_t device_bytes;   /* device memory owned by the handle */
    int32_t rows_per_block; /* row-gather launch shape in use: rows per block of the per-row
                               star kernel, -1 for the edge-fan kernel, 0 if unavailable */
    int32_t n_plans;        /* row-gather launch shapes available */
    int32_t persistent;     /* 1: the row gather runs as a persistent grid (a CTA's next block of
                               rows copies its column indices and walk while the current one
                               writes out), 0: one CTA per block of rows */
    int32_t exact_rows;     /* mixed modes: rows of the nodes of badly shaped elements
                               (|d1||d2||d3| > 16 |det| from any node); after every assembly or
                               time step these rows are recomputed in double from the coordinates
                               and overwritten (a float determinant of such an element carries
                               about that ratio times the float rounding of its edge vectors) */
    int32_t long_rows;      /* rows the row gather leaves out -- more than 32 entries (its walk
                               steps hold five bits of row position), or a star its walk
                               encoder could not cover -- computed after every row-gather
                               assembly or time step by one thread per row, in double; the rest
                               of the mesh stays on the row gather */
    int32_t fan_ok;         /* 1: the mesh has an edge-fan map (rows of at most 16 entries, the
                               ring of elements around every edge at most 7 nodes, no long
                               rows): the edge-fan kernel is available (nsi_set_launch) */
} NsiInfo;
nsi_status nsi_info(const NsiHandle* h, NsiInfo* info);

/*
 * Assemble A, G and rhs for the velocities in `f` (Section II-A, Listing 1)
 * using the handle's default scatter mode.  Device pointers; enqueues on
 * `stream`; overwrites every output entry.
 */
nsi_status nsi_assemble(NsiHandle* h, const NsiFields* f, const NsiOutputs* o, void* stream);

/* Same as nsi_assemble with an explicit scatter mode (nsi_scatter).  Paper:
 * the scatter of Listing 2 (perform_assembly_in_global_system), whose
 * conflicts shaped the FPGA design (Section III-B); the modes are this
 * library's ways of doing it on a GPU. */
nsi_status nsi_assemble_mode(NsiHandle* h, const NsiFields* f, const NsiOutputs* o, int32_t scatter,
                             void* stream);

/*
 * Assemble `count` independent meshes in one launch (one persistent grid
 * strides over every mesh's rows).  All handles must share one precision and
 * support the row-gather mode; count <= NSI_MAX_BATCH.  Pointers are passed to
 * the kernel by value, so the call is graph-capturable and allocates nothing.
 * (No counterpart in the paper, which assembles one mesh per call; the
 * per-mesh operation is nsi_assemble's.)
 */
#define NSI_MAX_BATCH 128
nsi_status nsi_assemble_batched(NsiHandle* const* hs, const NsiFields* fs, const NsiOutputs* os,
                                int32_t count, void* stream);

/*
 * One time step with cached geometry.  Over time steps on a fixed mesh with
 * fixed rho, mu and dt (Alya assembles every step, Section II), only the
 * convection and the RHS of the assembly depend on the velocity:
 *   A_val = A_static + C(u),  rhs = lumped rho u^n / dt  (as nsi_assemble),
 * where A_static is the A of nsi_assemble at u = 0 with the same rho, mu and
 * dt (the viscous part plus the lumped mass) and C(u) the convection term.  G
 * does not change and is not written.  A_static, A_val: device [nnz] of the
 * handle's output type (A_val may alias A_static: every entry is read before
 * it is written, by the same thread; both may be NULL when nnz = 0); rhs:
 * device [3][n_nodes], overwritten;
 * the velocities in `f` as for nsi_assemble.  Needs the row-gather map
 * (rows of at most 32 entries): NSI_ERR_UNSUPPORTED otherwise.
 */
nsi_status nsi_assemble_convective(NsiHandle* h, const NsiFields* f, const void* A_static, void* A_val,
                                   void* rhs, void* stream);

/*
 * The per-node outputs of the paper's assembly kernel
 * (perform_assembly_in_global_system, Listing 2), without the matrix:
 *   rhs[k][i]   = sum over elements e of i of rho |T_e| u^n_i[k] / (4 dt)  (rhsid)
 *   dt_rho[i]   = sum over elements e of i of rho |T_e| / (4 dt)           (dt_rho_nsi)
 *   mass_rho[i] = sum over elements e of i of rho |T_e| / 4                (mass_rho_nsi)
 * (the paper prints the accumulation, not the element values: read as the
 * row-sum lumped density mass over dt and the lumped density mass).  rhs:
 * device [3][n_nodes], dt_rho and mass_rho device [n_nodes], all of the
 * handle's output type and overwritten; u^n is f->u_n (or f->u).  Needs the
 * row-gather map: NSI_ERR_UNSUPPORTED otherwise.
 */
nsi_status nsi_assemble_nodal(NsiHandle* h, const NsiFields* f, void* rhs, void* dt_rho, void* mass_rho,
                              void* stream);

/*
 * The stabilised velocity block.  Paper Section II-A, Listing 4: the 12x12
 * element matrix of the velocity unknowns couples every pair of dimensions of
 * two nodes, equal dimensions receiving the scalar part; Table I's
 * calculate_tau_and_tim computes the stabilisation parameters, whose formulas
 * the paper does not print.  This library's reading: the Galerkin operator
 * above plus the implicit terms of Codina's algebraic subgrid scales
 * (Comput. Methods Appl. Mech. Engrg. 191 (2002) 4295-4321; linear elements,
 * c1 = 4, c2 = 2), per element
 *   tau1 = (4 mu / h^2 + 2 rho |ubar| / h)^-1,  tau2 = h^2 / (4 tau1),
 *   h = (6 |T_e|)^(1/3),  ubar = the mean of the element's four node velocities,
 *   Auu_e(a,i; b,j) = delta_ij ( A_e[a][b] + tau1 rho^2 int (u.grad N_a)(u.grad N_b) )
 *                   + mu int d_j N_a d_i N_b + tau2 int d_i N_a d_j N_b
 * (the SUPG convection product, the transposed-gradient half of the viscous
 * stress, the grad-div term of the pressure subscale).
 * Outputs (device, overwritten; double for NSI_FP64 and NSI_MIXED_F32_ACC64,
 * float for NSI_MIXED_F32_ACC32):
 *   Auu   [9][nnz]: component 3 i + j is the (i, j) entry of the 3x3 block
 *                   of every CSR entry (row node's dimension i, column
 *                   node's dimension j);
 *   G_val [3][nnz] and rhs [3][n_nodes]: as nsi_assemble.
 * One warp per row (or per two rows of at most 16 entries): each element of
 * the row's star is evaluated once, its contributions summed per entry in
 * element order (deterministic); rows of more than 32 entries
 * (NsiInfo.long_rows) and, in the mixed modes, the rows touching badly shaped
 * elements (NsiInfo.exact_rows) are then computed by one double-precision
 * thread per row.  Precision as nsi_assemble; in NSI_MIXED_F32_ACC64 an
 * entry's values are float sums of its edge's elements, and the diagonal
 * block (the lumped mass minus the row's other blocks) is formed from
 * compensated float-pair row totals.  The handle's scatter mode does not
 * apply.  NSI_ERR_UNSUPPORTED for meshes of more than 2^31 node-element
 * incidences.  Requires mu > 0 (tau1 of an element at rest is h^2 / (4 mu)),
 * rho >= 0, dt > 0 (NSI_ERR_INVALID_ARG otherwise).
 * Never allocates or synchronises.
 */
nsi_status nsi_assemble_stabilized(NsiHandle* h, const NsiFields* f, void* Auu, void* G_val, void* rhs,
                                   void* stream);

/*
 * Vector-Jacobian product of the assembled residual R(u, mu) = A(u) u - b
 * (b held fixed):  grad_u[l][m] = sum_{i,k} w[k][i] dR[k][i]/du[l][m] and
 * grad_mu = sum_{i,k} w[k][i] dR[k][i]/dmu.  Element geometry is recomputed
 * (no element matrices are stored).  w, grad_u: device [3][n_nodes] in the
 * handle's velocity type; grad_mu: device double scalar.  Both outputs are
 * overwritten.  (No counterpart in the paper: the derivative of the
 * Section II-A assembly with respect to the velocity and the viscosity.)
 */
nsi_status nsi_assemble_vjp(NsiHandle* h, const NsiFields* f, const void* w, void* grad_u,
                            double* grad_mu, void* stream);

/*
 * Residual of the assembled system without forming the matrix:
 * R[k][i] = sum_j A_ij u[k][j] - rhs[k][i] for the velocities in `f` (the
 * quantity whose adjoint nsi_assemble_vjp computes).  r: device [3][n_nodes]
 * in the handle's velocity type, overwritten.  (No counterpart in the
 * paper.)
 */
nsi_status nsi_residual(NsiHandle* h, const NsiFields* f, void* r, void* stream);

/*
 * End-to-end variant for callers holding HOST arrays: copies u (and u_n) from
 * host memory to handle-owned device staging, assembles, and copies A, G, rhs
 * back to the host buffers in `o` (pinned memory recommended), all on
 * `stream`, then synchronises it.  The first call allocates the staging
 * buffers; later calls reuse them.  Paper: the host-side movement of the
 * FPGA designs (Section III-B/C: the host streams element data to the card
 * and receives results over PCIe) has this call as its counterpart here.
 */
nsi_status nsi_assemble_host(NsiHandle* h, const NsiFields* f_host, const NsiOutputs* o_host,
                             void* stream);

/*
 * Allocation-free assembly, for callers that may not allocate device memory
 * while they run: code executing where cudaMalloc is not allowed or not
 * wanted, such as a plugin whose device memory budget is fixed when it is
 * loaded, a real-time loop that must not block on the allocator, or a host
 * that hands every allocation to its own memory manager.  (The paper has no
 * counterpart; this is an interface of this library only.)
 *
 * Same result as nsi_assemble in the row-gather mode, for a handle created
 * beforehand: the call runs the kernels nsi_assemble would run for the handle
 * (the star or edge-fan row gather chosen by nsi_set_launch or the autotuner,
 * the persistent grid, the bounds checks of a debug handle) and then, in the
 * mixed precisions, the double-precision rows of badly shaped elements.  The
 * call allocates nothing: the per-call node records go to a
 * scratch array compiled into the library (16 MiB, held by every GPU that
 * loads the library until the process exits), so meshes of at most 524,288
 * nodes in the mixed precisions and 262,144 nodes in FP64 are accepted;
 * larger ones return NSI_ERR_UNSUPPORTED with a message giving both sizes.
 * The first call on a device looks up the scratch's device address (one
 * cudaGetSymbolAddress, no allocation); make that first call before any stream
 * capture.  Every call on every handle shares the one scratch array and
 * rewrites all of it that it reads, so nothing needs clearing between calls,
 * but calls that overlap on the GPU (other streams, other threads) race on
 * it: serialise them.
 */
nsi_status nsi_assemble_noalloc(NsiHandle* h, const NsiFields* f, const NsiOutputs* o, void* stream);

/*
 * The exchange step of one mesh assembled by several ranks, each on a
 * disjoint set of its elements (paper Section III-C gives disjoint element
 * sets to concurrent engines; splitting one mesh over GPUs this way is this
 * library's design): each rank's assembly leaves partial sums in the rows of
 * nodes on the partition interfaces, and the rank owning such a node adds
 * the others' values into its row.  These two calls move and add values; the
 * partition, the ownership and the index maps are the caller's
 * (paper_2111_05651_gb300/partition.py builds them, and exchanges the
 * buffers with torch.distributed).
 *
 * nsi_gather_values: dst[k * ncomp + c] = src[c][idx[k]] for k < count, c <
 *   ncomp -- the values of the chosen entries of ncomp component arrays
 *   (device pointers, e.g. A and the three G arrays), packed row-major into
 *   the device buffer dst.
 * nsi_add_values: dst[c][idx[k]] += src[k * ncomp + c] -- packed values added
 *   into component arrays.  The idx of one call must be distinct (each
 *   position is read and written by one thread); the order of the additions
 *   is the order of the calls.
 * src/dst: host arrays of ncomp device pointers (1 <= ncomp <= 4); idx: device
 * int32 [count]; value_bytes: 8 (double) or 4 (float).  Enqueued on `stream`;
 * no allocation.  count = 0 does nothing.
 */
nsi_status nsi_gather_values(const void* const* src, int32_t ncomp, const int32_t* idx, int64_t count, void* dst,
                             int32_t value_bytes, void* stream);
nsi_status nsi_add_values(void* const* dst, int32_t ncomp, const int32_t* idx, int64_t count, const void* src,
                          int32_t value_bytes, void* stream);

/*
 * Synchronise `stream` and read the handle's device error word: NSI_OK, or
 * NSI_ERR_DEVICE_CHECK (bounds check fired; the word is then cleared).
 * (No counterpart in the paper.)
 */
nsi_status nsi_device_status(NsiHandle* h, void* stream);

/*
 * Launch autotuner (project-written): times every available launch choice on
 * this mesh with the given fields and outputs -- the row-gather kernel at each
 * rows-per-block shape that fits shared memory, the colouring kernel, the
 * atomic kernel with and without warp aggregation, and the edge-fan
 * row-gather kernel where the mesh has its map -- `reps` calls each after one
 * warm-up call, keeps the fastest as the handle's default, and reports it
 * (chosen_rows as in nsi_set_launch; 0 for colouring).
 * Synchronises `stream`; overwrites the outputs.  Either output may be NULL.
 * (No counterpart in the paper, whose FPGA designs were tuned by hand,
 * Section III.)
 */
nsi_status nsi_autotune(NsiHandle* h, const NsiFields* f, const NsiOutputs* o, int32_t reps, void* stream,
                        int32_t* chosen_scatter, int32_t* chosen_rows);

/*
 * Set the handle's default scatter mode and its kernel, e.g. to apply a cached
 * autotuning result.  With NSI_SCATTER_GATHER (or AUTO), rows_per_block > 0
 * selects the per-row star kernel with that many rows per block, -1 the
 * edge-fan kernel (one thread per CSR entry), 0 keeps the current choice.
 * With NSI_SCATTER_ATOMIC, rows_per_block 1 selects warp-aggregated atomics
 * (lanes adding to the same entry combine their values by shuffles and issue
 * one atomic), 2 one atomic per value (the default), 0 keeps the choice.
 * (Defined by this library's design; the paper's scatter is the host's.)
 */
nsi_status nsi_set_launch(NsiHandle* h, int32_t scatter, int32_t rows_per_block);

/*
 * Profiling hook: when both events (cudaEvent_t, created by the caller) are
 * non-NULL, every later assemble call on this handle records `start` right
 * before its main assembly kernel and `stop` right after it, on the call's
 * stream, so that the caller can time that kernel alone (the per-call node
 * packing and output zeroing stay outside the pair).  Pass NULLs to disable.
 * (No counterpart in the paper.)
 */
nsi_status nsi_set_timing_events(NsiHandle* h, void* start, void* stop);

/* Message describing the last failure on the calling thread ("" if none).
 * (No counterpart in the paper.) */
const char* nsi_last_error(void);

/* NSI_ABI_VERSION of the loaded library.  (No counterpart in the paper.) */
int32_t nsi_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NSI_ASSEMBLE_H */
