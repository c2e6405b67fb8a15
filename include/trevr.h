/*
 * trevr.h -- C ABI of the GB300 (sm_103a) implementation of the TREVR hot path.
 *
 * TREVR (Grond, Woods, Wadsley & Couchman 2019, arXiv:1902.08083) computes,
 * for every sink (gas particle), the angle-averaged intensity
 *
 *     F_p = sum over pseudo-sources C of  L_C exp(-tau_pC) / (4 pi s_pC^2)   (Eq. simpint)
 *
 * where the pseudo-sources come from a walk of a space-filling source tree
 * under the opening-angle criterion theta_open > l/r (Eq. openangle, Sec.
 * 2.2.1) and tau_pC is the optical depth of the reverse ray from the sink to
 * the pseudo-source, summed over tree cells (Eqs. taui, tausum, Sec. 2.2.2) and
 * refined into child cells where tau_ref < tau_max - tau_min (Eq. refcrit,
 * Sec. 2.2.3).
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers on the current CUDA device unless
 *     marked "host". The caller owns them; the library never frees them and
 *     never keeps them past the call (the tree copies what it needs).
 *   - Positions are structure-of-arrays: xyz points to 3*n floats laid out as
 *     x[0..n), y[0..n), z[0..n).
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream). Work is enqueued on it; see each function for when it syncs.
 *   - The return value is TREVR_OK (0) or one of the TREVR_ERR_* codes below.
 *     Errors found on the device (a point outside the domain, a non-finite
 *     input, a traversal stack overflow) are reported through a device status
 *     word read back at the function's sync point; the kernels never trap.
 *     Outputs are undefined when the return value is not TREVR_OK.
 *   - Particle and source counts are limited to 2^30 (indices are 32-bit).
 *   - Device memory: a tree's buffers, and the scratch of the tree build and of
 *     the adjoint, come from a stream-ordered memory pool the library creates on
 *     each device it is used on. The pool keeps memory that is freed (so that
 *     the next build or backward call reuses it without mapping it again) until
 *     the process exits.
 *   - Positions inside the library are relative to the domain's lower corner
 *     (x - lo), so fp32 rounding depends on the size of the domain, not on its
 *     distance from the origin; outputs that are positions say so.
 */
#ifndef TREVR_H
#define TREVR_H

#ifdef __cplusplus
extern "C" {
#endif

#define TREVR_OK 0
#define TREVR_ERR_INVALID_ARGUMENT 1 /* null pointer, bad size or parameter, NaN/negative input */
#define TREVR_ERR_OUT_OF_DOMAIN 2    /* a particle or source outside [lo, lo+side)^3 */
#define TREVR_ERR_STACK_OVERFLOW 3   /* a traversal stack would overflow (stack_depth too small) */
#define TREVR_ERR_ITERATION_LIMIT 4  /* a walk exceeded its iteration cap (hang guard) */
#define TREVR_ERR_CUDA 5             /* a CUDA runtime call failed */
#define TREVR_ERR_OUT_OF_MEMORY 6    /* device allocation failed */

typedef struct trevr_tree trevr_tree; /* opaque, device-resident, owned by the library */

/* Cubic domain: every particle and source must satisfy lo_d <= x_d < lo_d + side,
   evaluated in fp32. */
typedef struct {
    float lo[3];
    float side;
} trevr_domain;

/* The method's parameters (Sec. 2.2): theta_open (Eq. openangle, >= 0),
   tau_ref (Eq. refcrit; <= 0 means refine every cell down to the buckets) and
   the bucket size N_B (>= 1). The three tuning fields pick the launch shape of
   the sink walk; 0 selects the library default. */
typedef struct {
    float theta_open;
    float tau_ref;
    int bucket;
    int sinks_per_warp; /* sinks in each warp's chunk of the walk (a lane that finishes
                           its sink takes the next of the chunk); 0 = default (32) */
    int block_size;     /* threads per block of the walk, 0 = default */
    int stack_depth;    /* traversal stack entries per sink, 0 = default (64) */
    int walk_variant;   /* 1 = every lane walks its own sink; 2 = the 32 lanes of a warp
                           walk one shared stack and trace together the rays to a cell
                           they accept together; 3 = as 2, but each lane keeps its next
                           ray pending and the pending rays of all lanes (to different
                           cells) are traced together; 0 = default (3). All give the
                           same decisions and counters. */
    float bg_radius;    /* > 0: every source is a background source on the sphere of this
                           radius around the domain centre (Sec. 2.2.4), and a merged cell's
                           centre of luminosity is moved radially onto that sphere before
                           its ray is traced (the ray then ends in the leaf holding the
                           moved point). 0 = off. Only trevr_compute_flux accepts it. */
    float tau_stop;     /* > 0: early ray termination (Sec. 4, proposed there): a ray's
                           optical depth sum stops once it exceeds tau_stop, and the ray
                           then adds nothing (the flux drops by at most exp(-tau_stop)
                           times its unabsorbed value). The fp32 running sum decides.
                           0 = off; negative or NaN is an invalid argument. Only
                           trevr_compute_flux accepts it. */
    int sub_bucket;     /* 1: sub-bucket particle trace (Sec. 2.2.3, 3.1.3; needs
                           trevr_tree_set_smoothing). A leaf whose own particles ask for
                           refinement, (max - min of their alpha) * l > tau_ref (every
                           leaf if tau_ref <= 0), integrates the SPH field of the
                           particles along the ray's chord in it instead of using its
                           mean. The receiving particle is left out of that sum. 0 = off.
                           Only trevr_compute_flux accepts it, without bg_radius or
                           tau_stop. */
    int ray_walk;       /* 0: the paper's ray walk (Sec. 2.2.2, 3.1.3): the segments are
                           the sink's bucket S, the source cell C and the siblings of the
                           cells on the two paths up to their lowest common ancestor A,
                           each refined by Eq. refcrit. 1: the top-down ray walk that the
                           paper names as an alternative (Sec. 3.1.3, last paragraph of
                           "Refinement Criterion"; Sec. 4): the ray starts as the single
                           segment A and only Eq. refcrit splits it, so a ray costs one
                           segment where the medium has no spread of absorption. Its
                           segments are unions of the paper's walk's; tau_ref <= 0 gives
                           the same cells. Only trevr_compute_flux accepts 1, without
                           bg_radius, tau_stop or sub_bucket; it runs the merged-ray walk
                           (walk_variant 3). */
} trevr_params;

/* Totals over the sinks of one call, and timings (ms, CUDA events). */
typedef struct {
    long long interactions;      /* rays traced: accepted cells plus single sources */
    long long segments;          /* ray segments summed (cells whose mean absorption was used) */
    long long src_nodes_visited; /* source-tree cells tested against the opening angle */
    long long refine_expansions; /* cells replaced by their two children (Eq. refcrit) */
    long long cells_clipped;     /* ray/cell intersection tests (every cell record a ray read) */
    float build_ms;
    float walk_ms;
    long long rays_terminated;   /* rays cut off by tau_stop (of the interactions) */
    long long sub_bucket_segments; /* leaf segments integrated through the particles */
} trevr_stats;

/*
 * Build the radiation tree (Sec. 2.2, 2.3): Morton keys of the gas particles
 * (21 bits per axis, x most significant), a stable radix sort, the binary tree
 * of Morton prefixes with leaves of at most N_B particles (or of equal keys),
 * cut by planes so that the cells fill the domain; the sources deposited into
 * the leaves that hold them; and the cell moments: volume-weighted mean
 * absorption sum(w alpha)/sum(w) (Sec. 2.3, with w = m/rho this is
 * rho_cell = sum m / sum(m/rho) times kappa), the directional alpha_min /
 * alpha_max built bottom-up (Sec. 2.2.3), total luminosity and centre of
 * luminosity (Sec. 2.2.1).
 *
 *   gas_xyz  3*n_gas floats (SoA), gas particle positions; the sinks.
 *   alpha    n_gas floats, absorption coefficient alpha = kappa*rho >= 0.
 *   weight   n_gas floats > 0 (volume weight m/rho), or NULL for all 1.
 *   n_gas    1 .. 2^30.
 *   src_xyz  3*n_src floats (SoA), source positions.
 *   src_lum  n_src floats, luminosities >= 0.
 *   n_src    0 .. 2^30.
 *   dom      host pointer to the domain.
 *   prm      host pointer; only prm->bucket is used here.
 *   stream   cudaStream_t.
 *   out      host pointer; receives the tree (free with trevr_tree_free).
 * Synchronises `stream` before returning (the status word is read back).
 */
int trevr_build_tree(const float* gas_xyz, const float* alpha, const float* weight,
                     long long n_gas, const float* src_xyz, const float* src_lum, long long n_src,
                     const trevr_domain* dom, const trevr_params* prm, void* stream,
                     trevr_tree** out);

/*
 * Flux at the sinks (Eq. simpint summed over the pseudo-sources of the
 * opening-angle walk, Sec. 2.2.1-2.2.3), in fp32. Each sink's flux is a
 * compensated sum. The warp-shared walks (variants 2 and 3) sum a ray's optical
 * depth plainly, and the per-lane walk (variant 1) sums it with compensation.
 *
 *   t         tree from trevr_build_tree.
 *   sink_idx  n_sink int64 caller indices of gas particles, or NULL = all
 *             gas particles in the caller's order (then n_sink must be n_gas).
 *   prm       host pointer: theta_open, tau_ref, tuning fields.
 *   flux_out  n_sink floats: flux_out[k] is the flux at sink k.
 *   sink_counters  NULL, or 4*n_sink int32: per sink the number of rays,
 *             segments, source cells visited and refinements.
 *   stats     host pointer or NULL. When non-NULL the call synchronises the
 *             stream and fills the totals and walk time; when NULL the call
 *             is asynchronous and device errors surface at the next call
 *             that synchronises (trevr_check).
 */
int trevr_compute_flux(const trevr_tree* t, const long long* sink_idx, long long n_sink,
                       const trevr_params* prm, float* flux_out, int* sink_counters,
                       trevr_stats* stats, void* stream);

/*
 * Several bands (Sec. 4: many bands of radiation for a constant factor in cost).
 * Band b has its own absorption coefficient per particle and its own
 * luminosity per source. The bands share the walk and the rays. The tree, the
 * centres of luminosity and the opening-angle test use the band-summed
 * luminosity L_j = fp32(sum_b L_b,j), summed in FP64 in band order. Every band
 * sums its own optical depth (Eq. tausum) over the shared segments. A cell is
 * refined (Eq. refcrit) when any band asks for it, since its spread is
 * max_b (alpha_max,b - alpha_min,b). One band is the plain method.
 *
 *   alpha_bands  n_bands x n_gas floats, band-major (band b at b * n_gas),
 *                each >= 0 and finite.
 *   lum_bands    n_bands x n_src floats, band-major, each >= 0 and finite.
 *   n_bands      1 .. TREVR_MAX_BANDS.
 *   other arguments as in trevr_build_tree (band 0's alpha is checked there).
 * The tree holds 3 extra 16-byte records per cell and one per source. The
 * single-band calls (trevr_compute_flux and the rest, trevr_batch_create)
 * reject a tree with more than one band. Synchronises the stream.
 */
#define TREVR_MAX_BANDS 4
int trevr_build_tree_bands(const float* gas_xyz, const float* alpha_bands, const float* weight,
                           long long n_gas, const float* src_xyz, const float* lum_bands,
                           long long n_src, int n_bands, const trevr_domain* dom,
                           const trevr_params* prm, void* stream, trevr_tree** out);

/*
 * Smoothing lengths for the sub-bucket particle trace (Sec. 2.2.3, 3.1.3).
 * Below the buckets, the absorption is the SPH field
 * alpha(x) = sum_j alpha_j w_j W(|x - x_j|, h_j), where alpha_j w_j = kappa_j m_j
 * is particle j's absorbing mass. W is the cubic spline with support 2h:
 *   (1/(pi h^3)) (1 - 1.5 q^2 + 0.75 q^3)  for q = r/h < 1,
 *   (1/(pi h^3)) (2 - q)^3 / 4            for 1 <= q < 2,
 *   0                                     beyond.
 * The call lists, for every leaf, the particles whose support meets its box,
 * and keeps each leaf's alpha spread.
 *   hsml  n_gas floats on the device, caller order, each > 0 and finite.
 * Device memory grows by 20 B per particle, 8 B per cell, 24 B per
 * (leaf, neighbour) pair and 16 MiB for the tree's kernel-integral table. A
 * second call replaces the first. A tree with more than one band is rejected.
 * Synchronises the stream.
 */
int trevr_tree_set_smoothing(trevr_tree* t, const float* hsml, void* stream);

/*
 * Flux of every band at the sinks of a tree from trevr_build_tree_bands.
 *   flux_out   n_bands x n_sink floats, band-major: band b of the k-th sink at
 *              b * n_sink + k.
 *   other arguments as in trevr_compute_flux. The counters and stats are those
 *   of the shared walk. bg_radius and tau_stop must be 0. walk_variant is
 *   ignored: the bands use the merged-ray walk.
 * Synchronises the stream and reports device errors.
 */
int trevr_compute_flux_bands(const trevr_tree* t, const long long* sink_idx, long long n_sink,
                             const trevr_params* prm, float* flux_out, int* sink_counters,
                             trevr_stats* stats, void* stream);

/*
 * The flux and its next two direction moments at the sinks (Sec. 2.1: the
 * vector flux of Eq. simpflux, F = sum of L exp(-tau)/(4 pi s^2) n over the
 * pseudo-sources with n the unit vector from the pseudo-source to the sink, and
 * the radiation-pressure moment sum of the same terms times n n^T), from the
 * same walk, rays and decisions as trevr_compute_flux.
 *
 *   t, sink_idx, n_sink, prm  as in trevr_compute_flux (walk_variant ignored).
 *   flux_out  n_sink floats (Eq. simpint), as trevr_compute_flux.
 *   fvec_out  3*n_sink floats, SoA: x[0..n), y[0..n), z[0..n).
 *   press_out NULL or 6*n_sink floats, SoA in the order xx, yy, zz, xy, xz, yz
 *             (its trace equals flux_out).
 * Synchronises the stream and reports device errors.
 */
int trevr_compute_flux_moments(const trevr_tree* t, const long long* sink_idx, long long n_sink,
                               const trevr_params* prm, float* flux_out, float* fvec_out,
                               float* press_out, void* stream);

/*
 * Gradients of a scalar loss through the flux, with the decisions of the
 * forward pass held fixed (the merge/open choices of Eq. openangle, the
 * refinement choices of Eq. refcrit and the cells each ray touches): the
 * adjoint of Eq. simpint with tau from Eqs. taui/tausum. Centres of
 * luminosity move with the luminosities (c_C = sum L_j y_j / L_C, Sec.
 * 2.2.1); cell absorption is sum(w alpha)/sum(w) (Sec. 2.3).
 *
 *   t, sink_idx, n_sink, prm  exactly as in the forward call whose fluxes were
 *             differentiated (the walk is replayed with the same decisions).
 *   grad_flux  n_sink floats: dLoss/dF at each sink (same order as flux_out).
 *   grad_lum   n_src floats, caller order: dLoss/dL_j (overwritten).
 *   grad_alpha n_gas floats, caller order: dLoss/dalpha_i (overwritten).
 * Allocates its FP64 accumulators with cudaMallocAsync on `stream` and
 * synchronises the stream before returning. Gradients with respect to the
 * positions are not computed.
 */
int trevr_compute_flux_backward(const trevr_tree* t, const long long* sink_idx, long long n_sink,
                                const trevr_params* prm, const float* grad_flux, float* grad_lum,
                                float* grad_alpha, void* stream);

/*
 * Batched flux for many independent boxes (each its own tree) in ONE persistent
 * launch: the sinks of all trees are cut into work items of prm->sinks_per_warp
 * consecutive sinks (Morton order; a multiple of 32, 0 = 64), largest trees
 * first, and every warp of a grid of (SM count x resident blocks) takes the
 * next item from a device counter until none are left. Each sink's flux is the
 * same computation as trevr_compute_flux (Eq. simpint over the opening-angle
 * walk with tau_ref refinement), so the results are bit-identical to one plain
 * call per tree with the same parameters.
 *
 *   trevr_batch_create: trees = host array of n_trees tree handles (they must
 *             outlive the batch); uploads their views; synchronous.
 *   trevr_compute_flux_batched:
 *     prm       theta_open, tau_ref (all trees), sinks_per_warp (item size),
 *               block_size (64, 128 or 256; 0 = 128).
 *     flux_out  DEVICE array of n_trees device pointers; flux_out[b] receives
 *               n_gas(b) floats in that tree's caller order.
 *     stats     host pointer or NULL; non-NULL synchronises and fills totals.
 *   With stats == NULL the call only enqueues a memset and one kernel on
 *   `stream` (it can be captured in a CUDA graph once a first call with the
 *   same sinks_per_warp has built the work items; changing sinks_per_warp
 *   rebuilds them with a synchronous upload).
 *   trevr_batch_check: synchronise and return the batch's device status.
 */
typedef struct trevr_batch trevr_batch;
int trevr_batch_create(trevr_tree* const* trees, int n_trees, trevr_batch** out);
int trevr_compute_flux_batched(trevr_batch* batch, const trevr_params* prm,
                               float* const* flux_out, trevr_stats* stats, void* stream);
int trevr_batch_check(const trevr_batch* batch, void* stream);
void trevr_batch_free(trevr_batch* batch);

/* Synchronise `stream` and return the first device error recorded on the tree
   since the last check (TREVR_OK if none), clearing it. */
int trevr_check(const trevr_tree* t, void* stream);

/* Number of cells of the tree, the maximum cell depth, and the particle and
   source counts (host pointers, any may be NULL). */
int trevr_tree_info(const trevr_tree* t, long long* n_nodes, int* max_depth, long long* n_gas,
                    long long* n_src);

/*
 * Copy the tree out (for tests and tools). Node arrays are indexed by the
 * library's breadth-first cell numbering (root = 1, the children of a cell
 * are two consecutive cells 2k, 2k+1; entry 0 is unused), n_nodes+1 entries;
 * any pointer may be NULL. All are device pointers.
 *   key      n_gas uint64 Morton keys in sorted order;  perm n_gas int32 caller
 *            index of the i-th sorted particle;  leaf_of n_gas int32 leaf cell of
 *            the i-th sorted particle.
 *   first, count   int32 particle range of each cell in sorted order.
 *   child    int32 lower child (upper = child+1), -1 for a leaf.
 *   parent   int32 (0 for the root).   depth int32.
 *   glo, ghi 3 int32 per cell: integer box on the 2^21 grid, [glo, ghi).
 *   abar     fp32 mean absorption;  dalpha fp32 alpha_max - alpha_min;
 *   lum      fp32 total luminosity;  cen 3 fp32 centre of luminosity, relative to
 *            the domain's lower corner (the frame the walk computes in: x - lo);
 *   l2       fp32 squared distance from the centre to the furthest vertex.
 *   src_first, src_count  int32 range of each cell in the sorted sources;
 *   src_order n_src int32 caller index of the k-th sorted source.
 */
int trevr_tree_export(const trevr_tree* t, unsigned long long* key, int* perm, int* leaf_of,
                      int* first, int* count, int* child, int* parent, int* depth, int* glo,
                      int* ghi, float* abar, float* dalpha, float* lum, float* cen, float* l2,
                      int* src_first, int* src_count, int* src_order, void* stream);

/* Release the tree and every buffer it holds (synchronises the device). */
void trevr_tree_free(trevr_tree* t);

/*
 * Morton keys and stable sort of the gas particles WITHOUT any device
 * allocation. The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory while they run -- a host code
 * that reserves its device memory up front and forbids allocation inside its
 * time-step loop, or a plug-in that only receives buffers from the application
 * that owns the GPU. Its scratch memory is a fixed file-scope device array
 * sized for TREVR_NOALLOC_MAX_N particles (about 12.3 MiB, held on every GPU
 * that loads the library until the process exits).
 *
 * The result is the same as the keys and the permutation of trevr_build_tree
 * (see trevr_tree_export): Morton keys with 21 bits per axis, x most
 * significant, computed in fp32 from the domain, sorted stably.
 *
 *   gas_xyz   3*n_gas floats (SoA), device.
 *   n_gas     1 .. TREVR_NOALLOC_MAX_N; larger sizes return
 *             TREVR_ERR_INVALID_ARGUMENT without touching the GPU.
 *   dom       host pointer to the domain.
 *   keys_out  n_gas uint64, device: the keys in sorted order.
 *   perm_out  n_gas int32, device: caller index of the i-th sorted particle.
 *   stream    cudaStream_t. The call synchronises it before returning.
 * The first call on a device looks up the device address of the scratch array
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture. Every call shares the one array and overwrites it, so
 * calls whose work overlaps on the GPU (other streams or host threads) race.
 * The looked-up address is kept for the life of the process: after a
 * cudaDeviceReset of a device, do not call this function on that device again.
 * A point outside the domain returns TREVR_ERR_OUT_OF_DOMAIN.
 */
#define TREVR_NOALLOC_MAX_N (1 << 20)
int trevr_morton_sort_noalloc(const float* gas_xyz, long long n_gas, const trevr_domain* dom,
                              unsigned long long* keys_out, int* perm_out, void* stream);

/* Number of CUDA kernels this library has launched in the calling process
   (all devices, all streams); for launch accounting in benchmarks. */
unsigned long long trevr_kernel_launches(void);

/* Short English description of a status code (static storage). */
const char* trevr_status_string(int code);

#ifdef __cplusplus
}
#endif
#endif /* TREVR_H */
