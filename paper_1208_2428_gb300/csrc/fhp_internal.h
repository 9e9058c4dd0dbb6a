// fhp_internal.h -- layout and launcher declarations shared by the library's
// translation units (not part of the public ABI).
//
// Device layout of one lattice of W x H nodes (W multiple of 32, H even):
//   Wq = W / 32 words per row, nq = ceil(Wq / 4) quads of 4 words per row,
//   row pitch Pq = 4 * nq words (16-byte aligned rows; the words Wq..Pq-1 of
//   every row are padding and stay zero).  A plane is H * Pq words; a state
//   buffer is 7 consecutive planes (planes 0..5 movers along c_0..c_5,
//   plane 6 rest particles); the solid flags form one more plane.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace fhp {

struct Key2 {
    uint32_t lo, hi;
};

struct ForcingTable {
    unsigned long long q[33];
    // P + 1 with P = round(p * 2^32): Q_K <= K (P + 1), so u >= K (P + 1)
    // proves that none of K candidates is forced (cheap exact pre-check).
    unsigned long long p_plus_1;
};

struct Geometry {
    int W = 0, H = 0;
    int Wq = 0;         // words per row
    int nq = 0;         // quads per row
    int Pq = 0;         // row pitch in words (multiple of 4)
    size_t plane_words = 0;  // H * Pq
    int row_base = 0;   // lattice row of array row 0 (a strip of a larger lattice; even)
    int rules = 2;      // collision rule set: 2 = FHP-II, 1 = FHP-I, 3 = FHP-III (direct and ring kernels)
};

// Forcing thresholds of probability p (host): P = round-half-even(p * 2^32),
// computed from the integer and fraction parts of the exact double p * 2^32
// (independent of the floating-point rounding mode); S_0 = 2^32,
// S_g = floor(S_{g-1} (2^32 - P) / 2^32), Q_g = 2^32 - S_g (exact integers).
ForcingTable forcing_table(double p);

// Mask that enables the rest-particle rules of the bit-sliced scattering.
inline uint32_t rest_rules_mask(const Geometry& g) { return g.rules == 1 ? 0u : 0xFFFFFFFFu; }

Geometry make_geometry(int W, int H);

// Arguments of one k = 1 step kernel launch.
struct StepArgs {
    const uint32_t* __restrict__ src;    // 7 planes of S_t
    uint32_t* __restrict__ dst;          // 7 planes of S_{t+1}
    const uint32_t* __restrict__ solid;  // solid plane (read only if has_solid)
    unsigned long long plane_words;
    int H, Wq, nq, Pq;
    int rows_per_warp;       // nq < 32: rows of one parity packed into a warp
    int groups_per_parity;   // nq < 32: warps per row parity
    int warps_per_row;       // nq >= 32: warps covering one row
    Key2 key;
    uint32_t t_lo, t_hi;
    unsigned int* err;       // set nonzero if a bounded device-side wait gives up
    int y_base = 0;          // added to the row index that keys the random words (strips)
    uint32_t rest_rules = 0xFFFFFFFFu;  // ones: FHP-II rest-particle rules on; zero: FHP-I
    ForcingTable ft;
};

// Row tiling of the bulk-copy step kernel: tiles of R full rows, staged in a
// ring of shared-memory buffers by cp.async.bulk.
struct TileArgs {
    int R;                         // rows per tile
    int ntiles;                    // ceil(H / R)
    unsigned long long nq_magic;   // ceil(2^32 / nq): j / nq == (j * nq_magic) >> 32 for small j
};

// Step kernel choice: automatic, direct register loads, or the bulk-copy ring
// (cp.async.bulk into shared memory; falls back to direct when a row does not
// fit a stage).  Automatic picks the ring when it gets >= 2 tiles per SM.
// kStepRun: the ring kernel running many steps in one cooperative launch
// (per-tile dependency counters instead of a launch per step).
// kStepResident: lattices that fit in the SMs' shared memory stay on chip for
// all steps of a call (fhp_resident.cu).
enum StepKernel { kStepAuto = 0, kStepDirect = 1, kStepRing = 2, kStepRun = 3, kStepResident = 4 };

// Launch one time step (motion, scattering, bounce-back, forcing).
// `err` (device word, may be NULL) is set nonzero if a bounded wait gives up.
cudaError_t launch_step(const Geometry& g, const uint32_t* src, uint32_t* dst,
                        const uint32_t* solid, bool has_solid, bool force,
                        const ForcingTable& ft, Key2 key, uint64_t t, cudaStream_t stream,
                        unsigned int* err = nullptr, int kernel = kStepAuto);

// The kernel fhp_step uses for `requested`: kStepDirect, kStepRing or kStepRun
// (launch_step itself runs kStepRing for kStepRun: one step per launch).
int resolved_step_kernel(const Geometry& g, bool has_solid, int requested);

// Tiles of the ring / multi-step kernels (0 if a row does not fit a stage);
// the multi-step kernel needs that many counter words of scratch.
int run_tiles(const Geometry& g, bool has_solid);

// n >= 1 steps from buf0 (state at t0) in one cooperative launch; the result
// is in buf0 if n is even, else in buf1.  `done` holds run_tiles() words of
// scratch (zeroed by the call on the stream).
cudaError_t launch_run(const Geometry& g, uint32_t* buf0, uint32_t* buf1, const uint32_t* solid,
                       bool has_solid, bool force, const ForcingTable& ft, Key2 key, uint64_t t0,
                       int nsteps, unsigned int* done, cudaStream_t stream, unsigned int* err);

// Shared-memory resident lattices: supported when every SM's strip (one CTA
// per SM, at most one per row) fits in shared memory and the exchange rows fit
// the lattice's byte-staging area (`staging_bytes`).  `gh` is the number of
// steps between exchanges: 1 (each strip trades its edge rows every step) or
// 2 (each strip also computes 2 ghost rows per side itself and trades 2 rows
// every 2 steps; needs strips of at least 4 rows).  n >= 1 steps from buf0
// (state at t0); the result is in buf0 if n is even, else in buf1.  `halo`
// needs resident_halo_words() words, `flags` one word per SM (both scratch).
bool resident_supported(const Geometry& g, bool has_solid, size_t staging_bytes, int gh = 1);
size_t resident_halo_words(const Geometry& g, int gh);
cudaError_t launch_resident(const Geometry& g, uint32_t* buf0, uint32_t* buf1, const uint32_t* solid, bool has_solid,
                            bool force, const ForcingTable& ft, Key2 key, uint64_t t0, int nsteps, int gh,
                            uint32_t* halo, unsigned int* flags, cudaStream_t stream, unsigned int* err);

// Temporal blocking: k (2, 4 or 8) steps from src (state at t0) to dst in one
// pass.  Supported when rows are whole quads (W multiple of 128), there are
// at least 4 quads per row and H >= 2k + 2.
bool block_supported(const Geometry& g, int k);
cudaError_t launch_block(const Geometry& g, const uint32_t* src, uint32_t* dst, const uint32_t* solid,
                         bool has_solid, bool force, const ForcingTable& ft, Key2 key, uint64_t t0, int k,
                         cudaStream_t stream, unsigned int* err);

// Temporal blocking inside batches (fhp_batch_block.cu): one launch applies
// pass `pass` (k = 2 or 4 steps) to every member with more passes than that
// in the call, tile by tile over a list of (member, row tile) records.  A
// member's tile holds R_out full rows (even; batch_block_rows, 0 if the
// member's rows are too wide); the kernel stages R_out + 2k rows of the
// member's pitch in each of 16 shared-memory planes of kBBPlaneWords words.
constexpr int kBBPlaneWords = 3072;
struct BlockMember {
    StepArgs a;              // geometry, solid plane, key, forcing, rules, err (src, dst, t: set per pass)
    uint32_t* buf[2];        // state buffers; buf[cur] holds the state at step t0
    unsigned long long t0;   // the member's step at the start of the call
    int cur;
    int passes;              // blocked passes of the member in the call
    int R_out;               // output rows per tile
    int force;               // forcing probability nonzero
    int y0, rows_out, active;  // per tile: filled in by the kernel in its shared-memory copy
    int pad;
};
struct BlockTile {
    int lattice;             // index into the member table
    int tile;                // row tile of the member
};
int batch_block_rows(const Geometry& g, int k);
cudaError_t configure_batch_block();   // kernel attributes of the current device (first use loads the kernel)
cudaError_t launch_batch_block(const BlockMember* d_members, const BlockTile* d_tiles, int ntiles, int pass, int k,
                               unsigned int* err, cudaStream_t stream);

// Temporal blocking by row wavefronts (fhp_wave.cu): k (2, 3 or 4) steps from
// src (state at t0) to dst in one pass over full-width row bands, the
// intermediate levels in shared-memory row rings.  Supported when a row of
// every level ring fits shared memory (about W <= 16,384 for k = 2 and 3,
// 8,192 for k = 4) and the rule set is FHP-I or FHP-II.
bool wave_supported(const Geometry& g, int k);
cudaError_t launch_wave(const Geometry& g, const uint32_t* src, uint32_t* dst, const uint32_t* solid,
                        bool has_solid, bool force, const ForcingTable& ft, Key2 key, uint64_t t0, int k,
                        cudaStream_t stream, unsigned int* err);

// Pack H x W node bytes (device) into 7 state planes + the solid plane.
// Sets *device_any_solid to a nonzero value if any node is solid.
cudaError_t launch_pack(const Geometry& g, const uint8_t* bytes, uint32_t* state,
                        uint32_t* solid, unsigned int* device_any_solid, cudaStream_t stream);

// Generated initial state: bits 0..6 of every fluid node set independently
// with probability round(density * 2^16) / 2^16 from counter-based draws of
// the lattice seed (solid nodes end empty).
cudaError_t launch_init_random(const Geometry& g, uint32_t* state, const uint32_t* solid, bool has_solid,
                               uint64_t seed, double density, cudaStream_t stream);

// Unpack 7 state planes + the solid plane into H x W node bytes (device).
cudaError_t launch_unpack(const Geometry& g, const uint32_t* state, const uint32_t* solid,
                          uint8_t* bytes, cudaStream_t stream);

// Replace the solid plane from an H x W byte mask (nonzero = solid) and clear
// the particles of solid nodes in `state`.
cudaError_t launch_load_obstacles(const Geometry& g, const uint8_t* mask, uint32_t* state,
                                  uint32_t* solid, unsigned int* device_any_solid,
                                  cudaStream_t stream);

// Obstacles from shapes (kinds as FHP_SHAPE_*): replaces the solid plane and
// clears the particles of solid nodes.  *device_any_solid (may be NULL) is
// set nonzero if any node is solid.
struct Shape {
    int kind, a, b, c;
};
struct ShapeList {
    Shape s[8];
    int n;
};
cudaError_t launch_obstacle_shapes(const Geometry& g, const ShapeList& shapes, uint32_t* state, uint32_t* solid,
                                   unsigned int* device_any_solid, cudaStream_t stream);

// Coarse-grain over B x B blocks (B multiple of 32 dividing W and H).
cudaError_t launch_coarse_grain(const Geometry& g, const uint32_t* state, const uint32_t* solid,
                                bool has_solid, int B, int32_t* counts, float* rho, float* ux,
                                float* uy, cudaStream_t stream);

// Record the calling thread's last error (returned by fhp_last_error(NULL)).
void set_thread_error(const char* message);

// Philox4x32-10 over n counters (diagnostic entry point).
cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n,
                          cudaStream_t stream);

}  // namespace fhp
