/*
 * fhp.h -- C ABI of the GB300 FHP lattice-gas library (libfhp_gb300.so).
 *
 * The library advances a Frisch-Hasslacher-Pomeau lattice gas: a triangular
 * lattice whose nodes carry seven occupation bits (six moving directions and
 * one rest particle) plus a solid flag, updated by motion, scattering with
 * bounce-back on solid nodes, and horizontal momentum forcing
 * (Szkoda, Koza & Tykierko, arXiv:1208.2428, Section 2).
 *
 * Conventions shared by every call:
 *   - Node byte (paper Section 2, Fig. 1): bit i (i = 0..5) is a particle with
 *     velocity c_i at angle (i-2)*60 degrees (0 SW, 1 SE, 2 E, 3 NE, 4 NW,
 *     5 W), bit 6 is the rest particle, bit 7 marks a solid node.
 *   - Host lattice arrays are H x W bytes, row-major (row y, then x); row
 *     y = 0 is the bottom row and odd rows are shifted half a cell to the
 *     right (paper Section 2, Fig. 3).  W is a positive multiple of 32 and H
 *     is even and >= 2.  The lattice is periodic in x and y; walls are solid
 *     rows.
 *   - Every call returns an int status: FHP_OK (0) or one of the FHP_E*
 *     codes below.  No call aborts or throws; CUDA errors are captured and
 *     reported.  fhp_last_error() returns a message for the last failure.
 *   - Pointers named host_* are host memory owned by the caller; pointers
 *     named device_* are device memory of the lattice's device, owned by the
 *     caller.  The library never keeps a caller pointer after a call returns,
 *     except params->device_memory (see fhp_create).
 *   - Calls enqueue work on the lattice's stream.  Calls that read or write
 *     host buffers return only when the data is complete; calls taking
 *     device buffers are asynchronous with respect to the host.
 *   - A handle must not be used by two host threads at the same time.
 */
#ifndef FHP_GB300_H
#define FHP_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FHP_API __attribute__((visibility("default")))
#else
#define FHP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define FHP_OK 0
#define FHP_EINVAL 1   /* invalid argument (sizes, NULL pointers, ranges) */
#define FHP_ENOMEM 2   /* device or host allocation failed, or caller memory too small */
#define FHP_ECUDA 3    /* a CUDA runtime call failed */
#define FHP_ETIMEOUT 4 /* a bounded device-side wait gave up */
#define FHP_EBUSY 5    /* the object is in use */
#define FHP_EDEBUG 6   /* debug build: an index check failed (the access was skipped) */

typedef struct fhp_lattice fhp_lattice;

typedef struct fhp_params {
    int32_t width;              /* W: nodes per row; multiple of 32, >= 32 */
    int32_t height;             /* H: rows; even, >= 2 */
    uint64_t seed;              /* key of the counter-based random generator */
    double forcing_p;           /* forcing probability per candidate node, in [0, 1] */
    void* stream;               /* cudaStream_t to enqueue on; NULL = legacy default stream */
    void* device_memory;        /* optional caller-owned device memory, 256-byte aligned,
                                   at least fhp_required_bytes(W, H); NULL = library allocates */
    size_t device_memory_bytes; /* size of device_memory in bytes */
} fhp_params;

/* Bytes of device memory one lattice of W x H nodes uses: two bit-plane
 * state buffers (7 planes each), one solid plane, H counter words for the
 * multi-step kernel, and a staging area for transfers, coarse-grained
 * results and the resident kernel's exchange rows (W*H bytes, or 144 bytes
 * per row quad times min(H/4, 256) where that is larger, as it can be for
 * H < 1152).  Returns 0 for invalid sizes. */
FHP_API size_t fhp_required_bytes(int32_t width, int32_t height);

/* Create a lattice on the current CUDA device with all nodes empty and
 * fluid, at step t = 0.  If params->device_memory is not NULL the library
 * uses that memory and the caller must keep it alive until fhp_destroy;
 * otherwise the library allocates and frees its own.  On failure *out is set
 * to NULL and fhp_last_error(NULL) describes the error. */
FHP_API int fhp_create(fhp_lattice** out, const fhp_params* params);

/* Release the lattice and any memory the library allocated.  Waits for work
 * queued on the lattice's stream.  NULL is accepted and ignored. */
FHP_API void fhp_destroy(fhp_lattice* lattice);

/* Message for the last failed call on `lattice`, or, when `lattice` is NULL,
 * of the calling thread's last failed call that takes no lattice
 * (fhp_create, fhp_run_static, fhp_philox4x32_10_device).  Never NULL. */
FHP_API const char* fhp_last_error(const fhp_lattice* lattice);

/* Replace the whole lattice state, solid flags included (bit 7), from H x W
 * host bytes (paper Section 2, Fig. 1).  Particles on solid nodes are kept:
 * under bounce-back a solid node holds reflected particles for one step, so
 * a saved state round-trips exactly.  Synchronous. */
FHP_API int fhp_set_state(fhp_lattice* lattice, const uint8_t* host_bytes);

/* Copy the whole lattice state into H x W host bytes (same layout as
 * fhp_set_state).  Synchronous. */
FHP_API int fhp_get_state(fhp_lattice* lattice, uint8_t* host_bytes);

/* As fhp_set_state / fhp_get_state with H x W bytes in device memory of the
 * lattice's device.  fhp_get_state_device is asynchronous on the lattice's
 * stream; fhp_set_state_device returns once the state is packed, because it
 * reads back whether any node is solid (that selects the step kernel). */
FHP_API int fhp_set_state_device(fhp_lattice* lattice, const uint8_t* device_bytes);
FHP_API int fhp_get_state_device(fhp_lattice* lattice, uint8_t* device_bytes);

/* Replace the particles of every fluid node by a generated random state:
 * each of bits 0..6 set independently with probability
 * round(density * 2^16) / 2^16, drawn from Philox4x32-10 blocks with counter
 * (x / 32, y, bit, j) under the lattice seed's init key (seed halves xored
 * with 0x9E3779B9 and 0x7F4A7C15); node i = x mod 32 of a word takes block
 * j = i / 8, output word (i mod 8) / 2, the low 16 bits for even i.  Solid
 * nodes (load obstacles first) end empty.  Asynchronous. */
FHP_API int fhp_init_random(fhp_lattice* lattice, double density);

/* Replace the solid map from an H x W host mask (nonzero = solid) and clear
 * the particles of every node that is solid in the new map (paper Section 2:
 * boundary nodes carry bit 7 and reflect particles).  Synchronous. */
FHP_API int fhp_load_obstacles(fhp_lattice* lattice, const uint8_t* host_mask);

/* Advance the lattice by n >= 0 time steps.  One step is motion, then
 * scattering through the FHP-II rules with bounce-back on solid nodes, then
 * forcing (paper Section 2).  Random chirality and forcing draws depend only
 * on (seed, step, node), so results do not depend on how steps are grouped
 * into calls or kernel launches.  Asynchronous on the lattice's stream.
 * t + n must stay below 2^48. */
FHP_API int fhp_step(fhp_lattice* lattice, int64_t n);

/* Coarse-grain the current state over B x B blocks (B a multiple of 32 that
 * divides W and H).  For block (by, bx), at index c = by * (W/B) + bx:
 *   counts[9c + i], i = 0..6: fluid nodes of the block with bit i set;
 *   counts[9c + 7]: fluid nodes; counts[9c + 8]: particles on fluid nodes;
 *   rho[c] = mass / fluid nodes; ux[c] = jx2 / (2 mass);
 *   uy[c] = (sqrt(3)/2) jy / mass, with jx2 = sum_i n_i 2cos(theta_i) and
 *   jy = sum_i n_i sgn(sin(theta_i)); 0 where the denominator is 0.
 * Host buffers; any output may be NULL.  Synchronous. */
FHP_API int fhp_coarse_grain(fhp_lattice* lattice, int32_t block, int32_t* host_counts,
                     float* host_rho, float* host_ux, float* host_uy);

/* As fhp_coarse_grain with device buffers (none may be NULL).
 * Asynchronous on the lattice's stream. */
FHP_API int fhp_coarse_grain_device(fhp_lattice* lattice, int32_t block, int32_t* device_counts,
                            float* device_rho, float* device_ux, float* device_uy);

/* Current step counter t (number of steps applied since t = 0). */
FHP_API int64_t fhp_get_time(const fhp_lattice* lattice);

/* Set the step counter (for resuming a saved run); 0 <= t < 2^48. */
FHP_API int fhp_set_time(fhp_lattice* lattice, int64_t t);

/* Change the forcing probability (in [0, 1]) for subsequent steps. */
FHP_API int fhp_set_forcing(fhp_lattice* lattice, double p);

/* Number of steps fused into one kernel pass (temporal blocking): 1, 2, 3,
 * 4 or 8.  With k > 1, fhp_step runs passes that read the state from HBM
 * once, apply k steps on chip and write the result once.  Two kernels do it
 * (fhp_set_temporal_block_kernel chooses):
 *  - row wavefronts (k = 2, 3, 4) where a full row of every intermediate time
 *    level fits shared memory (FHP-I/II lattices up to about 16,384 nodes per
 *    row for k = 2 and 3, about 8,192 for k = 4): each CTA streams a band of
 *    whole rows through per-level row rings, recomputing only the k - 1 rows
 *    of each intermediate level beyond each band edge;
 *  - 2-D tiles (k = 2, 4, 8) elsewhere: a tile plus a halo of k rows and k
 *    words (forcing couples the 32 nodes of a word) is staged in shared
 *    memory (W a multiple of 128, at least 512 nodes per row, H >= 2k + 2).
 * Leftover steps (n mod k) and lattices neither kernel supports (and FHP-III
 * lattices) use the single-step kernels.  With step kernel 4 (resident) the
 * value is instead the number of steps between exchanges of strip rows: 2
 * selects the two-ghost-row variant where every strip holds at least 4 rows,
 * other values the one-row exchange.  Results are identical for every value.
 * Default 1. */
FHP_API int fhp_set_temporal_block(fhp_lattice* lattice, int32_t k);

/* Obstacles generated on the device from simple shapes (the walls and
 * cylinder of the paper's flows, Section 4), so no H x W mask crosses the
 * bus.  A node (x, y) (array indices) is solid if any shape covers it:
 *   FHP_SHAPE_DISC: (x - a)^2 + (y - b)^2 <= c^2;
 *   FHP_SHAPE_ROWS: a <= y < b (c unused).
 * Replaces the solid map and clears the particles of solid nodes, as
 * fhp_load_obstacles does with the equivalent mask.  At most
 * FHP_MAX_SHAPES shapes; FHP_EINVAL otherwise or for an unknown kind. */
#define FHP_SHAPE_DISC 1
#define FHP_SHAPE_ROWS 2
#define FHP_MAX_SHAPES 8
typedef struct fhp_shape {
    int32_t kind;
    int32_t a, b, c;
} fhp_shape;
FHP_API int fhp_load_obstacle_shapes(fhp_lattice* lattice, const fhp_shape* shapes, int32_t count);

/* Collision rule set (the paper's Fig. 2 is not legible; the default is
 * FHP-II).  FHP_RULES_FHP_II: two-body head-on collisions turned by +-60
 * degrees by the node's chirality bit, symmetric three-body collisions, and
 * rest-particle creation / annihilation (rest + c_i <-> c_{i-1} + c_{i+1}).
 * FHP_RULES_FHP_I: the original model without the rest-particle rules (a rest
 * particle, if present, is a spectator that never changes).
 * FHP_RULES_FHP_III: the collision-saturated set -- every fluid state that
 * shares its mass and momentum with another state changes: zero-momentum
 * states turn their movers by +-60 degrees (chirality), two-state classes
 * swap, and the three-state classes of momentum c_k cycle (chirality sets the
 * direction); it keeps every FHP-II collision.  FHP-III lattices step with
 * the direct, bulk-copy ring and multi-step ring kernels (step kernels 1-3;
 * the resident kernel and temporal blocks k > 1 fall back to those) and
 * cannot be batch members.  Takes effect from the next step.
 * FHP_EINVAL for other values. */
#define FHP_RULES_FHP_I 1
#define FHP_RULES_FHP_II 2
#define FHP_RULES_FHP_III 3
FHP_API int fhp_set_rules(fhp_lattice* lattice, int32_t rules);
FHP_API int fhp_get_rules(const fhp_lattice* lattice);

/* Row-strip decomposition of one lattice across devices (the paper's
 * multi-GPU runs, Table 1).  A strip is a lattice of its own whose array row
 * y is row row_base + y of the whole lattice: the row keys the random words,
 * so the strip's steps draw the whole lattice's chirality and forcing bits.
 * The strip still wraps periodically in its own rows; a caller keeps g ghost
 * rows above and below the rows it owns, refreshes them from the neighbouring
 * strips (fhp_get_rows_device / fhp_set_rows_device), and then advances at
 * most g steps, after which exactly the owned rows are exact.  row_base must
 * be even (odd rows keep their half-cell shift); default 0. */
FHP_API int fhp_set_row_offset(fhp_lattice* lattice, int32_t row_base);

/* Row pitch in 32-bit words (32 nodes per word, rows padded to 4 words), or
 * -1 for a NULL lattice. */
FHP_API int32_t fhp_row_pitch_words(const fhp_lattice* lattice);

/* Copy rows [y0, y0 + n) of the 7 state bit-planes to / from a device buffer
 * laid out [plane 0..6][row][word] (7 * n * pitch words, pitch from
 * fhp_row_pitch_words; padding words of a row are zero).  Asynchronous on the
 * lattice's stream; the buffer is the caller's and must stay valid until the
 * stream passes the copy.  FHP_EINVAL if the rows are outside the lattice. */
FHP_API int fhp_get_rows_device(fhp_lattice* lattice, int32_t y0, int32_t n, uint32_t* device_words);
FHP_API int fhp_set_rows_device(fhp_lattice* lattice, int32_t y0, int32_t n, const uint32_t* device_words);

/* Temporal block fhp_step will use (1 if blocking is off or unsupported for
 * this lattice; for the resident kernel the exchange interval, 1 or 2), or
 * -1 for a NULL lattice. */
FHP_API int fhp_get_temporal_block(const fhp_lattice* lattice);

/* Kernel of the temporally blocked passes: 0 = automatic (2-D tiles where
 * they support the lattice and k, else row wavefronts; default), 1 = row
 * wavefronts, 2 = 2-D tiles; a kernel that does not support the lattice or k
 * falls back to the other one.  Results are identical for every choice.
 * FHP_EINVAL for other values.  fhp_get_temporal_block_kernel returns the
 * kernel fhp_step will use for the current settings: 1 or 2, 0 when no
 * blocked pass runs (k = 1, or the resident kernel), -1 for NULL. */
FHP_API int fhp_set_temporal_block_kernel(fhp_lattice* lattice, int32_t kind);
FHP_API int fhp_get_temporal_block_kernel(const fhp_lattice* lattice);

/* Autotuner.  Times every step configuration that applies to this lattice --
 * direct, ring, multi-step and resident kernels (the resident one with
 * exchanges every step and every second step), and temporal blocks
 * k = 2, 3, 4, 8 --
 * over trial_steps steps each (a multiple of 8 in [8, 4096]; each candidate
 * runs once untimed, then timed with CUDA events on the lattice's stream) and
 * records the fastest for this device, lattice shape, rule set, and whether
 * the lattice has obstacles and forcing.  From then on every lattice of that
 * description whose settings are automatic (kernel 0, temporal block 1) runs
 * the recorded configuration.  The state and the step counter are those of
 * the call on return (the trials run from a saved copy of the state, which
 * takes a temporary device allocation of 7 planes).  Synchronous.  out_kernel
 * and out_temporal_block (may be NULL) receive the choice.  Results of
 * fhp_step are identical for every configuration. */
FHP_API int fhp_autotune(fhp_lattice* lattice, int32_t trial_steps, int32_t* out_kernel,
                         int32_t* out_temporal_block);

/* Step kernel used by fhp_step: 0 = automatic (default), 4 = shared-memory
 * resident (the lattice is cut into one strip per SM and stays in shared
 * memory for all steps of a call; only the strips' edge rows are exchanged
 * between steps -- for lattices whose strips fit, else as 0), 1 = direct (one
 * 128-node quad per thread, operands loaded into registers), 2 = bulk-copy
 * ring (persistent CTAs stage tiles of full rows in shared memory with
 * cp.async.bulk, one launch per step), 3 = multi-step ring (the ring kernel
 * running all steps of an fhp_step call in one cooperative launch, each tile
 * waiting only for the three tiles of the previous step it reads).  2 and 3
 * fall back to 1 when a row does not fit a stage; automatic picks 1 for
 * lattices of fewer than 8 tiles, 4 (with exchanges every second step where
 * the strips allow it) for lattices of fewer than 2 tiles per SM whose strips
 * fit, 3 up to 24 tiles per SM and 2 above (FHP-III lattices: never 4).
 * Results are identical for every choice.  While the kernel is automatic and the temporal block 1, a
 * configuration recorded by fhp_autotune for the lattice's description takes
 * precedence. */
FHP_API int fhp_set_step_kernel(fhp_lattice* lattice, int32_t kind);

/* The step kernel fhp_step will run for the lattice's current settings
 * (1, 2, 3 or 4), or -1 for a NULL lattice. */
FHP_API int fhp_get_step_kernel(const fhp_lattice* lattice);

/* Block the calling thread until all work queued on the lattice's stream
 * has finished; reports asynchronous CUDA errors, and FHP_ETIMEOUT if a step
 * kernel gave up waiting for its input copies (the state is then
 * unreliable). */
FHP_API int fhp_synchronize(fhp_lattice* lattice);

/* Number of kernel launches this lattice has issued since creation. */
FHP_API int64_t fhp_kernel_launches(const fhp_lattice* lattice);

/* Diagnostic (no counterpart in the paper): runs the library's two bounded
 * device-side wait helpers -- an mbarrier phase wait and a completion-counter
 * wait -- on conditions that never hold, on the current device.  Each gives
 * up after its limit (2 s), so the call takes about 4 s; *host_status gets
 * bit 0 if the barrier wait gave up and bit 1 if the counter wait did (3
 * when the timeout path works).  The device stays usable afterwards. */
FHP_API int fhp_selftest_wait_limits(uint32_t* host_status);


/* Diagnostic: Philox4x32-10 (Salmon et al., SC'11) evaluated by the
 * library's device code.  device_ctr holds n counters of 4 words,
 * device_key n keys of 2 words, device_out receives n blocks of 4 words.
 * Asynchronous on `stream` (cudaStream_t, NULL = legacy default stream). */
FHP_API int fhp_philox4x32_10_device(const uint32_t* device_ctr, const uint32_t* device_key,
                             uint32_t* device_out, int64_t n, void* stream);

/* ------------------------------------------------------------------------
 * Batches: many independent lattices advanced by shared kernel launches.
 *
 * A batch owns one device arena (library- or caller-allocated).  Members --
 * lattices of any size (W a multiple of 32 up to 32,768, H even), each with
 * its own seed, forcing probability, obstacles, step counter and optional
 * step budget -- are carved out of the arena and may be added or removed
 * between calls, while the others keep their state.  fhp_batch_step(n)
 * advances every member by min(n, its remaining budget) steps; each step is
 * one kernel launch over the tiles of all members (replayed from a captured
 * CUDA graph), or each pass of k steps one launch of the blocked kernel
 * (fhp_batch_set_temporal_block), and every member evolves exactly as it
 * would alone.
 * Slots are small integers, reused after fhp_batch_remove.  Calls on one
 * batch must not overlap in time.  Errors: FHP_EINVAL for bad slots or
 * arguments, FHP_ENOMEM when the arena cannot hold a new member (admission
 * control), FHP_ECUDA for CUDA failures; fhp_batch_last_error explains.
 * ------------------------------------------------------------------------ */
typedef struct fhp_batch fhp_batch;

/* Arena bytes one member of W x H nodes occupies (0 if it cannot be a
 * member).  Set/get state and coarse-graining briefly need W*H (resp. the
 * coarse fields) more, also taken from the arena. */
FHP_API size_t fhp_batch_lattice_bytes(int32_t width, int32_t height);

/* Create an empty batch with an arena of arena_bytes on the current device:
 * caller-owned if device_memory is not NULL (256-byte aligned, kept alive by
 * the caller until fhp_batch_destroy), else allocated by the library.  Work
 * is enqueued on `stream` (cudaStream_t, NULL = legacy default stream). */
FHP_API int fhp_batch_create(fhp_batch** out, size_t arena_bytes, void* device_memory, void* stream);
FHP_API void fhp_batch_destroy(fhp_batch* batch);
FHP_API const char* fhp_batch_last_error(const fhp_batch* batch);

/* Add an empty, all-fluid member at step 0 without a step budget; *slot
 * receives its slot.  FHP_ENOMEM if the arena has no room. */
FHP_API int fhp_batch_add(fhp_batch* batch, int32_t width, int32_t height, uint64_t seed, double forcing_p,
                          int32_t* slot);
/* Remove a member and return its memory to the arena (waits for queued work). */
FHP_API int fhp_batch_remove(fhp_batch* batch, int32_t slot);
/* As fhp_batch_remove without waiting: the block returns to the arena at
 * once and any later use of it is queued on the batch's stream behind the
 * work already there.  Work the caller queued on other streams that reads the
 * member (fhp_batch_coarse_grain_device) must have finished. */
FHP_API int fhp_batch_remove_async(fhp_batch* batch, int32_t slot);

/* Generated initial state of a member (as fhp_init_random). */
FHP_API int fhp_batch_init_random(fhp_batch* batch, int32_t slot, double density);
/* Obstacles of a member from shapes (as fhp_load_obstacle_shapes);
 * asynchronous on the batch's stream. */
FHP_API int fhp_batch_load_obstacle_shapes(fhp_batch* batch, int32_t slot, const fhp_shape* shapes, int32_t count);
/* Collision rule set of a member (as fhp_set_rules; FHP_RULES_FHP_I or
 * FHP_RULES_FHP_II -- FHP-III runs on single lattices only, FHP_EINVAL). */
FHP_API int fhp_batch_set_rules(fhp_batch* batch, int32_t slot, int32_t rules);
/* Obstacles of a member (as fhp_load_obstacles), H x W bytes, nonzero =
 * solid.  Asynchronous: the mask is copied on the batch's stream; a pageable
 * buffer may be reused on return, a page-locked one only after
 * fhp_batch_synchronize.  FHP_ENOMEM if the arena has no room for the H x W
 * staging bytes. */
FHP_API int fhp_batch_load_obstacles(fhp_batch* batch, int32_t slot, const uint8_t* host_mask);

/* Member state as H x W node bytes (as fhp_set_state / fhp_get_state). */
FHP_API int fhp_batch_set_state(fhp_batch* batch, int32_t slot, const uint8_t* host_bytes);
FHP_API int fhp_batch_get_state(fhp_batch* batch, int32_t slot, uint8_t* host_bytes);
FHP_API int fhp_batch_set_time(fhp_batch* batch, int32_t slot, int64_t t);
FHP_API int64_t fhp_batch_get_time(const fhp_batch* batch, int32_t slot);

/* Step budget of a member: fhp_batch_step advances it by at most this many
 * more steps (-1 = no budget, the default). */
FHP_API int fhp_batch_set_steps_left(fhp_batch* batch, int32_t slot, int64_t steps);
FHP_API int64_t fhp_batch_get_steps_left(const fhp_batch* batch, int32_t slot);

/* Advance every member by min(n, its budget) steps.  Asynchronous. */
FHP_API int fhp_batch_step(fhp_batch* batch, int64_t n);

/* Batch step kernels.  SINGLE_STEP: one launch of the batch kernel per step
 * (replayed from captured CUDA graphs, see fhp_batch_set_graph_steps).
 * MULTI_STEP: all steps of an fhp_batch_step call in one cooperative launch;
 * a tile is staged for step s once the tiles of step s - 1 it reads (itself
 * and its two neighbours in its lattice) are finished, tracked by per-tile
 * counters.  AUTO (default): autotuned online together with the tile size
 * and the temporal block -- batches are classed by the binary order of
 * magnitude of their tile count at the default size of 256 quads (128-node
 * units) per tile; the first call in a class of at least
 * c * max(16, graph steps) steps runs an equal part of its steps (rounded
 * down to a multiple of 4) with each of c candidates -- both kernels; while
 * the tile size is automatic (fhp_batch_set_tile_quads), tiles of 256 and of
 * 128 quads; while the temporal block is automatic, blocked passes of 2 and
 * of 4 steps (c = 6 with both automatic) -- timed with CUDA events on the
 * batch's stream after the one-time set-up of every candidate (graph
 * capture, device tables, kernel attributes), and a later call records the
 * candidate with the most node updates per millisecond for the class (read
 * without waiting); until then SINGLE_STEP with 256-quad tiles and no
 * blocking runs.  Results are identical for every choice. */
#define FHP_BATCH_KERNEL_AUTO 0
#define FHP_BATCH_KERNEL_SINGLE_STEP 1
#define FHP_BATCH_KERNEL_MULTI_STEP 2
FHP_API int fhp_batch_set_step_kernel(fhp_batch* batch, int32_t kind);
FHP_API int fhp_batch_get_step_kernel(const fhp_batch* batch);
/* The kernel AUTO has recorded for batches of `ntiles` tiles at the default
 * tile size (0: the batch's current members): 0 = not yet measured, else
 * SINGLE_STEP or MULTI_STEP; -1 for invalid arguments.
 * fhp_batch_get_tuned_tile_quads: the tile size recorded with it (0 = not
 * yet measured). */
FHP_API int fhp_batch_get_tuned_kernel(const fhp_batch* batch, int32_t ntiles);
FHP_API int fhp_batch_get_tuned_tile_quads(const fhp_batch* batch, int32_t ntiles);
/* Tile size of the batch kernels' work lists in quads (4 words, 128 nodes)
 * per tile: 64, 128 or 256 (each tile whole rows of one member, at most 32
 * KB of planes), or 0 = automatic (default: tuned online with the kernel,
 * see above).  Results are identical for every size.
 * fhp_batch_get_tile_quads returns the size of the current tile list. */
FHP_API int fhp_batch_set_tile_quads(fhp_batch* batch, int32_t quads);
FHP_API int fhp_batch_get_tile_quads(const fhp_batch* batch);
/* Number of row tiles of the current members (the unit of the batch
 * kernels' work lists); -1 on error. */
FHP_API int32_t fhp_batch_tile_count(fhp_batch* batch);

/* Temporal blocking inside batches (the paper's kernels run one step per
 * pass over the lattice; this is an alternative order of the same updates).
 * With k = 2 or 4, each fhp_batch_step call advances every member whose rows
 * are narrow enough (fhp_batch_block_rows > 0) by floor(s / k) passes of k
 * steps, s = min(n, its budget): one launch per pass over tiles of full rows
 * of all such members, each tile staged in shared memory with k extra rows
 * above and below (periodic), stepped k times there and stored once.  The
 * remaining steps (s mod k, all s for wider members) run on the batch step
 * kernel.  Every member's state equals s single steps bit for bit.
 * k = 1: no blocking.  k = 0 (default): automatic -- while the step kernel is
 * AUTO, blocked passes of k = 2 and k = 4 (remainders on the single-step
 * kernel) join the online tuning trial as two more candidates (c = 6, or 4
 * with a fixed tile size) and the fastest candidate's temporal block is
 * recorded with its kernel; otherwise none.  FHP_EINVAL for other values.
 * Blocked passes take a descriptor table (about 0.4 KB per member slot) and
 * a tile list (12 bytes per tile) from the arena: with k = 2 or 4 a call
 * fails with FHP_ENOMEM if the arena cannot hold them; the automatic choice
 * then tunes without the blocked candidates.
 * fhp_batch_get_tuned_temporal_block: the block recorded for batches of
 * `ntiles` tiles (0 = the current members; 0 = not yet measured, -1 for
 * invalid arguments). */
FHP_API int fhp_batch_set_temporal_block(fhp_batch* batch, int32_t k);
FHP_API int fhp_batch_get_temporal_block(const fhp_batch* batch);
FHP_API int fhp_batch_get_tuned_temporal_block(const fhp_batch* batch, int32_t ntiles);
/* Output rows per blocked tile of a W x H member at temporal block k (2 or
 * 4): the largest even R, at most H, whose R + 2k staged rows fit one staged
 * plane of 3,072 words (a row is W / 32 words rounded up to a multiple of 4);
 * 0 if the member takes no blocked passes: R would be below 4k (and below
 * H), k is not 2 or 4, or the sizes are invalid. */
FHP_API int fhp_batch_block_rows(int32_t width, int32_t height, int32_t k);

/* Steps per captured CUDA graph of batch launches (0: launch directly).  The
 * graph reads the tile list and its length from device memory, so it is
 * captured once and survives members joining and leaving (it is captured
 * again only when the descriptor tables grow). */
FHP_API int fhp_batch_set_graph_steps(fhp_batch* batch, int32_t steps);

/* Coarse-grain one member into device buffers ([H/B][W/B][9] int32 counts,
 * [H/B][W/B] float rho, ux, uy; all required) on the caller's `stream`
 * (cudaStream_t, NULL = legacy default), asynchronously.  It reads the
 * member's current state: the caller orders the stream after the work that
 * produced it (for example an event recorded on the batch's stream after the
 * step call) and keeps later steps of the member from overlapping (a member
 * whose step budget is spent is not touched by fhp_batch_step). */
FHP_API int fhp_batch_coarse_grain_device(fhp_batch* batch, int32_t slot, int32_t block, int32_t* device_counts,
                                          float* device_rho, float* device_ux, float* device_uy, void* stream);

/* Coarse-grain one member into host buffers (as fhp_coarse_grain). */
FHP_API int fhp_batch_coarse_grain(fhp_batch* batch, int32_t slot, int32_t block, int32_t* host_counts,
                                   float* host_rho, float* host_ux, float* host_uy);

/* Wait for queued work; FHP_ETIMEOUT if a batch kernel gave up waiting. */
FHP_API int fhp_batch_synchronize(fhp_batch* batch);
FHP_API int32_t fhp_batch_count(const fhp_batch* batch);
FHP_API size_t fhp_batch_free_bytes(const fhp_batch* batch);
FHP_API int64_t fhp_batch_kernel_launches(const fhp_batch* batch);

/* Size in bytes of the device array that fhp_run_static works in. */
#define FHP_STATIC_SCRATCH_BYTES (16u << 20)

/* fhp_run_static: advance a lattice by n steps without allocating any device
 * memory.  This entry point has no counterpart in the paper; it exists for
 * callers that cannot allocate device memory -- plugins whose host
 * application owns all GPU memory through its own pool, services with a hard
 * device-memory cap fixed at start-up, and latency-critical loops where an
 * allocation, which may synchronise the device, is not acceptable.
 *
 * device_bytes_in / device_bytes_out: H x W node bytes (same layout as
 * fhp_set_state, solid flags in bit 7) in device memory of the current
 * device, owned by the caller; they may be the same buffer.  The run starts
 * at step t0 with the generator key `seed` and forcing probability
 * `forcing_p`, and gives exactly the state that fhp_create + fhp_set_state +
 * fhp_set_time(t0) + fhp_step(n) + fhp_get_state would give.  Asynchronous
 * on `stream` (cudaStream_t, NULL = legacy default stream).
 *
 * All intermediate data (two bit-plane state buffers, the solid plane, a flag
 * word) live in one file-scope __device__ array of FHP_STATIC_SCRATCH_BYTES
 * bytes, which every GPU that loads the library holds until the process
 * exits.  The call calls no cudaMalloc, cudaFree or other allocating routine.
 * Limit: 15 bit-planes of the lattice (rows padded to 128 nodes) plus 256
 * bytes must fit, i.e. up to about 8.9 million nodes (4096 x 2048 fits,
 * 4096 x 4096 does not); larger lattices fail with FHP_EINVAL.
 * The first call on a device looks the array's device address up
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  The address is kept for the device's context
 * and looked up again if that context was destroyed and made again
 * (cudaDeviceReset).  Steps run on the direct step kernel, which has no
 * device-side waits, so nothing can time out unseen in this asynchronous
 * call.  Every call on a device shares the array and it
 * keeps the previous call's contents (the call rewrites all of it that it
 * reads, and clears the flag word); calls whose GPU work overlaps -- from
 * different streams or host threads -- race on it and must be serialised by
 * the caller.  On failure fhp_last_error(NULL) describes the error. */
FHP_API int fhp_run_static(const uint8_t* device_bytes_in, uint8_t* device_bytes_out, int32_t width,
                           int32_t height, uint64_t seed, int64_t t0, int64_t n, double forcing_p,
                           void* stream);

/* ------------------------------------------------------------------------
 * Debug build (the library compiled with -DFHP_DEBUG: libfhp_gb300_debug.so).
 * Its kernels check every index that addresses a lattice plane, a staged
 * tile or a shared-memory ring against the buffer's extent before the
 * access; a failing check skips the access and records the check's site in
 * the kernel's error word, which fhp_synchronize / fhp_batch_synchronize
 * report as FHP_EDEBUG.  Every region of a lattice's or batch member's
 * device memory is followed by a 256-byte canary block.  No check traps.
 * ------------------------------------------------------------------------ */

/* 1 in the debug build, 0 in the release build. */
FHP_API int fhp_debug_build(void);

/* Compare the lattice's canary blocks with their fill (synchronous):
 * *checked = blocks compared (0 in the release build, which has none),
 * *corrupted = blocks whose bytes changed. */
FHP_API int fhp_debug_canaries(fhp_lattice* lattice, int32_t* checked, int32_t* corrupted);

/* As fhp_debug_canaries for every member of a batch. */
FHP_API int fhp_batch_debug_canaries(fhp_batch* batch, int32_t* checked, int32_t* corrupted);

/* Debug build: run one index check that fails on purpose and guards no
 * access, and return the error word it left (kErrBounds bit 1 and its site
 * code 99 in bits 8..15).  Shows that failing checks are recorded.
 * FHP_EINVAL in the release build.  Synchronous; allocates one word. */
FHP_API int fhp_debug_selftest(uint32_t* host_word);

#ifdef __cplusplus
}
#endif

#endif /* FHP_GB300_H */
