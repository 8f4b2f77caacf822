/*
 * sg.h -- C ABI of libsg, the GB300 (sm_103a) hot path for embedded
 * Sierpinski-gasket domains.
 *
 * Method: C. A. Navarro, B. Bustos, R. Vega, N. Hitschfeld, "Block-space GPU
 * Mapping for Embedded Sierpinski Gasket Fractals", arXiv:1706.04552.
 *
 * Domain.  Level r (0 <= r <= 16), side n = 2^r.  A grid is a dense
 * row-major n x n array in device memory, pitch n elements: cell (x, y)
 * (column x, row y) lives at index y*n + x.  The gasket G_r is the set of
 * cells with (x & y) == 0; it has 3^r cells (Section III-A).  The paper draws
 * the same set mirrored vertically (x & (n-1-y) == 0, Section III-D).
 *
 * Block space.  A tile ("block" in the paper) is a rho x rho square of cells,
 * rho = 2^s, 1 <= rho <= 64, rho <= n.  The tiles form an n_b x n_b box,
 * n_b = n / rho; exactly 3^(r-s) of them hold gasket cells, and each of those
 * holds the level-s gasket (3^s cells).
 *
 * Maps (how parallel work is assigned to tiles and cells):
 *   SG_MAP_LAMBDA         the paper's lambda(omega) (Theorem 1): a parallel
 *                         space of 3^(r-s) tiles, each decoded to its block
 *                         coordinate with a warp reduction over the base-3
 *                         digits of omega; inside a tile every slot is
 *                         visited and tested (bounding sub-box, Section
 *                         III-D, the variant the paper measured).
 *   SG_MAP_BBOX           bounding box: the identity map over all n_b^2
 *                         tiles, every cell tests membership (Section I).
 *   SG_MAP_LAMBDA_LUT     lambda for tiles; inside a tile only the 3^s member
 *                         slots are visited, in the row-major order of the
 *                         paper's shared lookup table (Section III-D, Shared
 *                         Lookup Table); each thread computes the entries it
 *                         visits once and keeps them in registers.  Write
 *                         pass only.
 *   SG_MAP_LAMBDA_UNROLL  lambda for tiles; inside a tile each thread applies
 *                         lambda again to its own index (Section III-D,
 *                         Further Unrolling).  Write pass only.
 *
 * Conventions for every call:
 *   - Ownership: the caller owns all memory.  libsg never allocates, frees or
 *     keeps a pointer after the call returns.
 *   - Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).
 *     Kernel calls are asynchronous on it and never synchronise the host.
 *   - Errors: arguments are checked on the host before any launch; a bad
 *     argument returns SG_EINVAL and launches nothing.  A failed launch
 *     returns SG_ECUDA (the CUDA error text is available from
 *     sg_last_error_string()).  Nothing is thrown and nothing exits.
 *   - Device: the current CUDA device of the calling thread.
 *   - Thread safety: calls may be made from several host threads at once.
 */
#ifndef SG_H
#define SG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SG_ABI_VERSION 2

/* Exported from libsg.so (the library is built with hidden visibility). */
#if defined(__GNUC__)
#define SG_API __attribute__((visibility("default")))
#else
#define SG_API
#endif

typedef enum {
    SG_OK = 0,
    SG_EINVAL = 1,        /* an argument is out of range, null or misaligned */
    SG_ECUDA = 2,         /* the CUDA runtime reported an error */
    SG_ENOMEM = 3,        /* reserved: libsg itself never allocates */
    SG_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
    SG_EUNSUPPORTED = 5   /* valid arguments, combination not provided */
} sg_status;

typedef enum { SG_U8 = 0, SG_F32 = 1 } sg_dtype;

typedef enum {
    SG_MAP_LAMBDA = 0,
    SG_MAP_BBOX = 1,
    SG_MAP_LAMBDA_LUT = 2,
    SG_MAP_LAMBDA_UNROLL = 3
} sg_map;

/* Order in which the lambda block space Pi is walked.  lambda(omega) itself
 * is the same in both; only which tile a given launch index q names differs.
 *   SG_ORDER_ROWMAJOR:    omega = (q mod 3^floor(rb/2), q div 3^floor(rb/2)),
 *                         the paper's two-dimensional grid row by row.
 *   SG_ORDER_INTERLEAVED: the base-3 digits of q are dealt alternately to
 *                         omega_y (digits 0, 2, 4, ...) and omega_x (digits
 *                         1, 3, 5, ...), so digit mu-1 of q is beta_mu and
 *                         consecutive q are neighbouring tiles. */
typedef enum { SG_ORDER_ROWMAJOR = 0, SG_ORDER_INTERLEAVED = 1 } sg_order;

/* How the write pass stores (see sg_map_write). */
typedef enum {
    SG_STORE_AUTO = 0,      /* the library's choice for dtype and rho */
    SG_STORE_SCATTER = 1,   /* one store per gasket cell */
    SG_STORE_STAGED = 2,    /* whole 16-byte chunks merged in shared memory;
                               needs rho * element size >= 16 bytes */
    SG_STORE_TMA = 3,       /* whole tiles moved by 2-D bulk tensor copies (TMA),
                               several tiles in flight per team; same
                               requirement as SG_STORE_STAGED */
    SG_STORE_FILL = 4,      /* write-only: every tile that holds gasket cells is
                               written whole, v(x, y) at gasket cells and 0 at
                               the other cells of the tile; nothing is read.
                               The result equals the other modes' whenever the
                               grid is 0 off the gasket (the zero matrix of the
                               paper's benchmark, the stencils' invariant).
                               Same requirement as SG_STORE_STAGED. */
    SG_STORE_SECTOR = 5,    /* write-only, one lane per 32-cell-wide unit: every
                               32-byte sector that holds gasket cells is written
                               whole with one 32-byte store, v(x, y) at gasket
                               cells and 0 at its other cells; nothing is read.
                               Equal to the preserving modes whenever the grid is
                               0 off the gasket.  Needs rho * element size >= 32
                               bytes and a 32-byte aligned grid. */
    SG_STORE_MERGE = 6,     /* as SG_STORE_SECTOR, but each such sector is read
                               (32-byte load), its gasket cells replaced and
                               written back; off-gasket cells keep their content
                               (no other kernel may write the grid meanwhile).
                               Same requirements. */
    SG_STORE_MASKED = 7     /* as SG_STORE_SECTOR, but only the gasket cells are
                               stored (one 4-, 2- or 1-byte store per run of
                               gasket cells in a 32-bit word, one store per cell
                               for float32); the L2 completes each sector from
                               DRAM.  Only gasket cells ever change.  Same
                               requirements. */
} sg_store;

/* Launch options of the *_ex calls.  Zero-initialise, then set fields. */
typedef struct {
    int order;          /* sg_order; -1 = library default */
    int store;          /* sg_store: the write pass's store path; for sg_ca_step_ex
                           and sg_diffuse_step_ex (and their k = 1 forms),
                           SG_STORE_TMA stages each tile and its halo with one
                           2-D bulk tensor copy instead of 16-byte chunk copies
                           (CA at rho = 32, 64; diffusion at rho = 16, 32;
                           other tile sides SG_EUNSUPPORTED); other values are
                           ignored by the stencils */
    int ctas_per_sm;    /* CTAs per SM of the persistent grid; 0 = occupancy maximum */
    int reserved[5];    /* must be 0 */
} sg_launch_opts;

typedef enum {
    SG_VAL_CONST = 0,     /* u8: low 8 bits of value_or_seed; f32: low 32 bits
                             reinterpreted as an IEEE float */
    SG_VAL_LINEAR31 = 1,  /* (x*31 + y) & 0xFF (as float for f32) */
    SG_VAL_HASH = 2       /* h = SplitMix64 output for state
                             (seed * 0x9E3779B97F4A7C15) XOR (y*n + x);
                             u8: h >> 56; f32: (h >> 40) * 2^-24 */
} sg_value_kind;

/*
 * sg_map_write -- the map-and-write pass (Section IV): every gasket cell of
 * the level-r grid receives v(x, y); every other cell keeps its content.
 *
 *   r              level, 0..16
 *   rho            tile side, a power of two in 1..64, rho <= 2^r
 *   map            any sg_map
 *   dtype          element type of `grid` (1 or 4 bytes)
 *   grid           device pointer to n*n elements (f32: 4-byte aligned)
 *   value_kind     how v(x, y) is formed (see sg_value_kind)
 *   value_or_seed  the constant, or the hash seed
 *   stream         cudaStream_t
 * Launches one kernel.  Returns SG_OK, SG_EINVAL or SG_ECUDA.
 *
 * The default (SG_STORE_AUTO) is SG_STORE_MERGE where rho * element size >= 32
 * bytes and `grid` is 32-byte aligned, else SG_STORE_STAGED where rho *
 * element size >= 16 bytes and `grid` is 16-byte aligned, else
 * SG_STORE_SCATTER.  With SG_STORE_MERGE, SG_STORE_STAGED or SG_STORE_TMA the
 * off-gasket cells of a touched sector or tile are read and written back
 * unchanged, so no other kernel may write `grid` while the pass runs; with
 * SG_STORE_SCATTER only gasket cells are ever stored.  SG_STORE_FILL (on request only) writes 0 to
 * the off-gasket cells of every tile that holds gasket cells.  SG_STORE_SECTOR,
 * SG_STORE_MERGE and SG_STORE_MASKED (on request only) move whole 32-byte
 * sectors with one lane per unit (see sg_store).
 */
SG_API sg_status sg_map_write(int r, int rho, sg_map map, sg_dtype dtype, void *grid,
                              sg_value_kind value_kind, uint64_t value_or_seed,
                              void *stream);

/*
 * sg_ca_step -- one step of the Life-like B3/S23 automaton restricted to the
 * gasket (the nearest-neighbour simulations that motivate the embedded
 * layout, Section I): a gasket cell is alive next iff exactly 3 of its 8
 * in-grid gasket neighbours are alive, or it is alive and exactly 2 are.
 * The grid border does not wrap.
 *
 *   in, out  device pointers to n*n uint8 states, 16-byte aligned, distinct
 *            and not overlapping.  Precondition: `in` holds 0 or 1 on gasket
 *            cells and 0 off the gasket; `out` holds 0 off the gasket.
 *            Postcondition: `out` holds the next state on every gasket cell
 *            and 0 off the gasket (so in/out can be swapped and stepped
 *            again).  Buffers zero-filled once satisfy both conditions.
 *   map      SG_MAP_LAMBDA or SG_MAP_BBOX (others: SG_EUNSUPPORTED)
 * Each tile is staged in shared memory with its halo; tiles are written
 * whole (off-gasket cells inside a non-empty tile are written as 0).
 * Launches one kernel.
 */
SG_API sg_status sg_ca_step(int r, int rho, sg_map map, const uint8_t *in,
                            uint8_t *out, void *stream);

/*
 * sg_diffuse_step -- one explicit FP32 diffusion step on the gasket's
 * 4-neighbour graph: for a gasket cell with in-grid gasket 4-neighbours N,
 * u' = u + alpha * (sum_{j in N} u_j - |N| * u).  Off-gasket cells stay 0.
 * (The paper names nearest-neighbour simulations in general, Section I; the
 * update rule is the one stated for this library.)
 *
 *   in, out  device pointers to n*n floats, 16-byte aligned, distinct.
 *            Precondition: `in` is 0 off the gasket and `out` is 0 off the
 *            gasket; postcondition as for sg_ca_step.
 *   alpha    step weight; the update is a convex combination for
 *            0 <= alpha <= 0.25.  Any finite value is accepted.
 *   map      SG_MAP_LAMBDA or SG_MAP_BBOX
 * Launches one kernel.
 */
SG_API sg_status sg_diffuse_step(int r, int rho, sg_map map, const float *in,
                                 float *out, float alpha, void *stream);

/* sg_map_write / sg_ca_step / sg_diffuse_step with launch options (NULL =
 * defaults).  A store mode the tile shape cannot use returns SG_EUNSUPPORTED;
 * a bad option value returns SG_EINVAL. */
SG_API sg_status sg_map_write_ex(int r, int rho, sg_map map, sg_dtype dtype, void *grid,
                                 sg_value_kind value_kind, uint64_t value_or_seed,
                                 const sg_launch_opts *opts, void *stream);
SG_API sg_status sg_ca_step_ex(int r, int rho, sg_map map, const uint8_t *in, uint8_t *out,
                               const sg_launch_opts *opts, void *stream);
SG_API sg_status sg_diffuse_step_ex(int r, int rho, sg_map map, const float *in, float *out,
                                    float alpha, const sg_launch_opts *opts, void *stream);

/*
 * sg_map_write_mapped -- the map-and-write pass on a grid that stays in host
 * memory.  host_grid is page-locked host memory mapped into the device's
 * address space (cudaHostAlloc, or pinned torch tensors, on a system with
 * unified addressing); the kernel reads and writes it where it is, over the
 * host link (NVLink-C2C on Grace), so only the touched chunks cross it: no
 * staging copy of the whole grid is made.  The pointer is checked with
 * cudaPointerGetAttributes before any launch (other memory: SG_EINVAL).
 * Stores: SG_STORE_AUTO (merge for tile rows of >= 32 bytes on a 32-byte
 * aligned grid, else staged where the tile rows allow it, else scatter),
 * SG_STORE_STAGED, SG_STORE_SCATTER, or SG_STORE_FILL: here the 32-byte
 * sectors that hold gasket cells are written whole with plain stores (0 at
 * their off-gasket cells) and nothing is read, so only the writes cross the
 * link -- equal to the others on a grid that is 0 off the gasket.
 * The sector modes (SG_STORE_SECTOR, SG_STORE_MERGE, SG_STORE_MASKED) run as on
 * a device grid, with 32-byte plain loads and stores over the link (tile rows
 * of 32 bytes and a 32-byte aligned grid).  SG_STORE_TMA (bulk tensor copies)
 * is SG_EUNSUPPORTED here.  The allocation must hold
 * the whole n*n grid (its size cannot be queried; a shorter one is the
 * caller's error, as for a device grid).  Otherwise as sg_map_write_ex; the
 * result is in host memory once the stream has completed.
 */
SG_API sg_status sg_map_write_mapped(int r, int rho, sg_map map, sg_dtype dtype,
                                     void *host_grid, sg_value_kind value_kind,
                                     uint64_t value_or_seed, const sg_launch_opts *opts,
                                     void *stream);

/*
 * sg_ca_steps / sg_diffuse_steps -- k consecutive steps of sg_ca_step /
 * sg_diffuse_step in one launch: out = step^k(in); `in` is not modified.
 * Every tile is staged in shared memory with a halo at least k cells deep
 * (rounded up to 4, 8 or 16 rows and to whole 16-byte chunks across), the k
 * steps run there, and only the tile is written back, so HBM sees the tile
 * bytes about once in and once out per launch rather than per step.  Each
 * cell's arithmetic is that of the single step, so the result equals k
 * calls of the single step.  (The paper fuses nothing; the per-tile lambda
 * map is that of Theorem 1.)
 *
 *   k        1 .. SG_FUSE_MAX; k = 1 runs the single-step kernel
 *   rho      16, 32 or 64 (other tile sides: SG_EUNSUPPORTED)
 *   in, out, map, alpha, preconditions and postconditions: as for the
 *            single step.
 * Launches one kernel.
 */
#define SG_FUSE_MAX 16
SG_API sg_status sg_ca_steps(int r, int rho, sg_map map, const uint8_t *in, uint8_t *out,
                             int k, const sg_launch_opts *opts, void *stream);
SG_API sg_status sg_diffuse_steps(int r, int rho, sg_map map, const float *in, float *out,
                                  float alpha, int k, const sg_launch_opts *opts,
                                  void *stream);

/*
 * sg_block_map -- the lambda block decode on its own (Theorem 1: Eq. beta,
 * Eq. Delta, Eq. tau, Eq. lambda), for checking the map bit for bit.
 * For every launch index q in [0, 3^rb), omega(q) as `order` defines it
 * (sg_order); (bx[q], by[q]) = (lambda_x(omega), 2^rb - 1 - lambda_y(omega)),
 * i.e. the paper's lambda mirrored into the (x & y) == 0 orientation.
 * bx, by: device arrays of 3^rb uint32.  rb: 0..16.  Launches one kernel.
 */
SG_API sg_status sg_block_map(int rb, sg_order order, uint32_t *bx, uint32_t *by,
                              void *stream);

/*
 * sg_launch_stats -- host-only accounting of one pass (Lemma 1, Theorem 2):
 * `launched` = cell slots the map's threads examine (lambda sub-box:
 * 3^(r-s) * rho^2; bounding box: n^2; lookup table / unrolling: 3^r),
 * `useful` = gasket cells = 3^r.  No GPU work.  Either pointer may be NULL.
 */
SG_API sg_status sg_launch_stats(int r, int rho, sg_map map, uint64_t *launched,
                                 uint64_t *useful);

/* ------------------------------------------------------------------------
 * Batches: many gaskets of uneven levels stepped by one launch.
 *
 * A batch is `count` gaskets, gasket i of level levels[i] with its own pair
 * of uint8 CA state buffers (buf_a[i], buf_b[i]; n_i*n_i bytes each, 16-byte
 * aligned, same conditions as sg_ca_step).  A step runs one persistent grid
 * over a single work list -- the concatenation of every gasket's lambda block
 * space, 3^(r_i - s) tiles each, indexed through a prefix sum -- instead of
 * one grid per gasket.  Parity 0 reads buf_a and writes buf_b; parity 1 the
 * reverse.  Results are bit-identical to stepping each gasket alone with
 * sg_ca_step.  The paper has no counterpart for batching; the per-gasket work
 * is the same lambda map (Theorem 1) and stencil as sg_ca_step.
 * ------------------------------------------------------------------------ */

/* A planned batch (filled by sg_batch_ca_plan; plain data the caller owns). */
typedef struct {
    void *workspace;            /* device memory holding the work list */
    uint64_t workspace_bytes;
    int count;                  /* gaskets */
    int rho;                    /* tile side: 16, 32 or 64 */
    uint32_t total_tiles;       /* work items per step */
    uint32_t max_level;
    int reserved[4];
} sg_batch_plan;

/* Device bytes the work list of `count` gaskets needs (0 if count is out of
 * range 1..65535).  Host-only. */
SG_API uint64_t sg_batch_workspace_bytes(int count);

/* Build the work list in `workspace` (caller-owned device memory of at least
 * sg_batch_workspace_bytes(count) bytes, 16-byte aligned) and fill *plan.
 * Every level must satisfy log2(rho) <= level <= 16.  levels, buf_a and buf_b
 * are host arrays of `count` entries (buf_* hold device pointers); they are
 * copied before the call returns.  One host-to-device copy on `stream`. */
SG_API sg_status sg_batch_ca_plan(int count, const int *levels, uint8_t *const *buf_a,
                                  uint8_t *const *buf_b, int rho, void *workspace,
                                  uint64_t workspace_bytes, sg_batch_plan *plan, void *stream);

/* One CA step of every gasket of the batch: one launch. */
SG_API sg_status sg_batch_ca_step(const sg_batch_plan *plan, int parity,
                                  const sg_launch_opts *opts, void *stream);

/* Capture `steps` consecutive batch steps (parities start_parity,
 * start_parity ^ 1, ...) into an instantiated CUDA graph (*graph, a
 * cudaGraphExec_t).  Launch it with sg_graph_launch, release it with
 * sg_graph_destroy.  The plan's workspace and buffers must outlive it. */
SG_API sg_status sg_batch_ca_graph_create(const sg_batch_plan *plan, int steps,
                                          int start_parity, const sg_launch_opts *opts,
                                          void **graph);
SG_API sg_status sg_graph_launch(void *graph, void *stream);
SG_API sg_status sg_graph_destroy(void *graph);

/* k fused steps of every gasket of the batch in one launch (k = 1 .. SG_FUSE_MAX;
 * k = 1 is sg_batch_ca_step): parity 0 reads buf_a and writes k steps later
 * into buf_b, parity 1 the reverse, as for sg_ca_steps.  A warp takes one
 * work item at a time and runs its tile's k steps bit-sliced in shared
 * memory; results equal k single batch steps. */
SG_API sg_status sg_batch_ca_steps(const sg_batch_plan *plan, int parity, int k,
                                   const sg_launch_opts *opts, void *stream);

/* Capture `steps` steps as launches of k fused steps (the last launch takes
 * the remainder), parities alternating from start_parity: after
 * ceil(steps / k) launches the state is in buf_a if that count is even
 * (start_parity 0).  Otherwise as sg_batch_ca_graph_create. */
SG_API sg_status sg_batch_ca_graph_create_fused(const sg_batch_plan *plan, int steps, int k,
                                                int start_parity, const sg_launch_opts *opts,
                                                void **graph);

/* Autotune a batch: time `trial_steps` parity-0 steps for every rho in
 * {16, 32, 64} allowed by the smallest level, both walking orders and
 * CTAs per SM in {occupancy maximum, 2, 4, 8}; plan the batch with the
 * fastest rho and return its launch options.  Parity-0 steps only read
 * buf_a, so the batch's current state (in buf_a) is left as it was; buf_b is
 * overwritten.  Results are cached per multiset of levels for the process.
 * Synchronises `stream`. */
SG_API sg_status sg_batch_ca_autotune(int count, const int *levels, uint8_t *const *buf_a,
                                      uint8_t *const *buf_b, void *workspace,
                                      uint64_t workspace_bytes, int trial_steps,
                                      sg_batch_plan *plan, sg_launch_opts *opts_out,
                                      void *stream);

/* sg_batch_ca_autotune for launches of k fused steps (sg_batch_ca_steps):
 * times `trial_launches` parity-0 launches of k steps per candidate (buf_a is
 * left as it was; buf_b is overwritten). */
SG_API sg_status sg_batch_ca_autotune_fused(int count, const int *levels, uint8_t *const *buf_a,
                                            uint8_t *const *buf_b, void *workspace,
                                            uint64_t workspace_bytes, int trial_launches, int k,
                                            sg_batch_plan *plan, sg_launch_opts *opts_out,
                                            void *stream);

/*
 * sg_batch_ca_step_noalloc -- one batch step for callers that cannot allocate
 * device memory.  The paper has no counterpart: this is a library
 * convenience.
 *
 * Who needs it: code that must not allocate device memory at the moment it
 * steps a batch -- a real-time loop that fixed its memory budget at start-up,
 * a plugin whose host application owns every device allocation, a server
 * that has already given all of HBM to its own pool.  There a cudaMalloc (or
 * any allocating library call, torch's included) can fail, stall the device
 * or break the host's accounting.  This call allocates nothing: the work list
 * that sg_batch_ca_plan would put in a caller-provided workspace lives in a
 * fixed array inside libsg instead, sized for SG_NOALLOC_MAX_GASKETS gaskets
 * (about 24 KB; every GPU that loads the library keeps it until the process
 * exits).  The caller still provides the gaskets' state buffers.
 *
 * Arguments as for sg_batch_ca_plan plus a sg_batch_ca_step parity; each
 * call rebuilds the work list (one host-to-device copy on `stream`) and then
 * launches the step, with results identical to sg_batch_ca_step.
 *   - More than SG_NOALLOC_MAX_GASKETS gaskets: SG_EINVAL, with the reason in
 *     sg_last_error_string().
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and keeps it for the life of the process; calls
 *     after a cudaDeviceReset of that device are not supported.
 *   - Each call copies the work list from a host buffer inside libsg that the
 *     next call overwrites, so it returns SG_EUNSUPPORTED while `stream` is
 *     being captured, before it copies or launches anything.
 *   - Every call shares the one array, and it keeps the last call's contents.
 *     Calls whose copies and kernels can overlap on the GPU (for example on
 *     two streams without ordering between them) race on it: order them on
 *     one stream or with events.
 */
#define SG_NOALLOC_MAX_GASKETS 1024
SG_API sg_status sg_batch_ca_step_noalloc(int count, const int *levels, uint8_t *const *buf_a,
                                          uint8_t *const *buf_b, int rho, int parity,
                                          const sg_launch_opts *opts, void *stream);

/*
 * Compact layout (the succinct blocked layout of Section II, with the
 * block-space map of Theorem 1 as the order of its blocks).  A compact array
 * at level r and tile side rho = 2^s holds only the 3^r gasket cells:
 * element i holds cell (bx*rho + tx, by*rho + ty), where (bx, by) is the
 * lambda block of launch index q = i div 3^s in the walking order
 * opts->order (the same block sg_block_map lists at position q), and
 * (tx, ty) is the (i mod 3^s)-th cell of the level-s gasket read row by row
 * (rows top to bottom, each row left to right).  Every non-empty tile holds
 * that same pattern (Section III), so the tiles are runs of 3^s consecutive
 * elements.  At r = 16 an 8-bit array takes 43 MB instead of 4.3 GB.
 *
 * Common arguments and errors:
 *   r, rho   as for sg_map_write (rho a power of two in 1..64, rho <= 2^r)
 *   opts     NULL or launch options: order and ctas_per_sm are used; store
 *            must be SG_STORE_AUTO (other values: SG_EUNSUPPORTED)
 *   compact arrays: device pointers to 3^r elements, aligned to the
 *            element size; embedded grids: device pointers to n*n elements
 *            (n = 2^r), aligned to the element size
 *   stream   cudaStream_t; every call launches one kernel and returns
 *            without synchronising
 * SG_EINVAL for out-of-range values, null or misaligned pointers, or an
 * output that is also the input; SG_ECUDA if the launch failed.
 */

/* sg_compact_pack -- compact[i] = grid at the cell of element i.  Reads only
 * gasket cells of `grid`. */
SG_API sg_status sg_compact_pack(int r, int rho, sg_dtype dtype, const void *grid,
                                 void *compact, const sg_launch_opts *opts, void *stream);

/* sg_compact_unpack -- grid at the cell of element i = compact[i].  Writes
 * only gasket cells of `grid`; every other cell keeps its content. */
SG_API sg_status sg_compact_unpack(int r, int rho, sg_dtype dtype, const void *compact,
                                   void *grid, const sg_launch_opts *opts, void *stream);

/* sg_compact_map_write -- the map-and-write pass (Section IV) on a compact
 * array: element i receives v(x, y) of its cell (sg_value_kind, the same
 * values sg_map_write writes there). */
SG_API sg_status sg_compact_map_write(int r, int rho, sg_dtype dtype, void *compact,
                                      sg_value_kind value_kind, uint64_t value_or_seed,
                                      const sg_launch_opts *opts, void *stream);

/* sg_compact_map_write_mapped -- sg_compact_map_write on a compact array
 * in page-locked host memory mapped into the device's address space
 * (cudaHostAlloc / cudaHostRegister with mapping; on Grace-Blackwell the
 * kernel writes it over NVLink-C2C).  The array is written once, as whole
 * consecutive sectors; nothing is read.  Other memory: SG_EINVAL before any
 * launch.  The values are in host memory once `stream` has completed. */
SG_API sg_status sg_compact_map_write_mapped(int r, int rho, sg_dtype dtype, void *host_compact,
                                             sg_value_kind value_kind, uint64_t value_or_seed,
                                             const sg_launch_opts *opts, void *stream);

/* sg_compact_ca_step -- one gasket-restricted B3/S23 step on compact 0/1
 * states: out = pack(sg_ca_step(unpack(in))), cell for cell.  in != out. */
SG_API sg_status sg_compact_ca_step(int r, int rho, const uint8_t *in, uint8_t *out,
                                    const sg_launch_opts *opts, void *stream);

/* sg_compact_ca_steps -- k CA steps in one launch on compact 0/1 states
 * (temporal blocking): out = the state after k sg_compact_ca_step calls, bit
 * for bit.  Each 64-tile is stepped k times in shared memory with the cells
 * of its neighbouring tiles that k steps can reach.  k in 1 ..
 * SG_FUSE_MAX (k = 1 is sg_compact_ca_step); rho must be 64 for k > 1
 * (SG_EUNSUPPORTED otherwise).  in != out. */
SG_API sg_status sg_compact_ca_steps(int r, int rho, int k, const uint8_t *in, uint8_t *out,
                                     const sg_launch_opts *opts, void *stream);

/* sg_compact_diffuse_step -- one explicit diffusion step on a compact field:
 * out = pack(sg_diffuse_step(unpack(in))), bit for bit (the same arithmetic
 * per cell).  in != out; alpha finite. */
SG_API sg_status sg_compact_diffuse_step(int r, int rho, const float *in, float *out,
                                         float alpha, const sg_launch_opts *opts,
                                         void *stream);

/*
 * sg_device_status -- report and clear the device status word of the current
 * device.  Kernels with bounded waits (SG_STORE_TMA, sg_wait_selftest) record
 * a wait that gave up there instead of spinning; the call synchronises
 * `stream` and returns SG_ETIMEOUT if any kernel recorded one since the last
 * call, else SG_OK (or SG_ECUDA if the status could not be read).  The fused
 * diffusion kernel for rho = 32, 64 records a unit whose live chunks exceed
 * the bound its registers are sized for (proved on the host never to happen);
 * that is reported as SG_EUNSUPPORTED.
 */
SG_API sg_status sg_device_status(void *stream);

/*
 * sg_wait_selftest -- exercise, without any fault, the bounded device-side
 * wait that the SG_STORE_TMA kernels use (failure detection; no operation of
 * the paper).  Launches `blocks` blocks of 128 threads on `stream`
 * (asynchronous).  Each block initialises a shared-memory mbarrier that
 * expects one arrival, and all its threads wait on it, bounded by `limit_ns`
 * nanoseconds of %globaltimer time and by a poll count.
 *   - arrive != 0: one thread arrives, the wait completes, nothing is recorded.
 *   - arrive == 0: nothing ever arrives; every wait gives up after about
 *     limit_ns, the kernel records SG_ETIMEOUT in the device status word
 *     (read and cleared by sg_device_status) and returns normally.  The CUDA
 *     context stays usable.
 * Errors: SG_EINVAL for `blocks` outside [1, 1024] or `limit_ns` outside
 * [1000, 2000000000] (2 s is the limit of the product kernels' waits);
 * SG_ECUDA if the launch failed.
 */
SG_API sg_status sg_wait_selftest(int blocks, int arrive, uint64_t limit_ns, void *stream);

/* Human-readable name of a status code (static storage). */
SG_API const char *sg_status_str(sg_status status);

/* Text of the last CUDA error seen by a libsg call on this host thread
 * ("" if none).  Static thread-local storage, valid until the next call. */
SG_API const char *sg_last_error_string(void);

/* SG_ABI_VERSION of the loaded library. */
SG_API int sg_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SG_H */
