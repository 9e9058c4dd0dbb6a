// fhp_debug.cuh -- index checks of the debug build (compiled with -DFHP_DEBUG).
//
// Compute-sanitizer is not available where this library is tested, so the
// debug build of the library checks, in device code, every index that
// addresses a lattice plane, a staged tile or a shared-memory ring against
// the extent of its buffer before the access.  A failing check does not trap:
// it sets kErrBounds and the check's site code (bits 8..15) in the kernel's
// error word, and the access is skipped; the host reports FHP_EDEBUG from
// fhp_synchronize (or fhp_batch_synchronize).  In the release build every
// check is the constant true and costs nothing.
#pragma once

#include <cstdint>

namespace fhp {

constexpr unsigned int kErrBounds = 2u;   // error-word bit of a failed debug check (bit 0: a wait gave up)

// Site codes (bits 8..15 of the error word) of the checks.
enum DebugSite : unsigned int {
    kSiteStoreQuad = 1,      // global store of a result quad (row, quad)
    kSiteStageFit = 2,       // a tile's planes fit its shared-memory stage
    kSiteIssueTile = 3,      // bulk-copy source row and destination rows of a tile
    kSiteStageQuad = 4,      // staged words a quad reads (row in tile, word in row)
    kSiteDirectQuad = 5,     // direct kernel loads (rows y-1, y, y+1; words)
    kSiteWaveSmem = 6,       // wavefront rings within the dynamic shared memory
    kSiteWaveQuad = 7,       // wavefront ring words a quad reads or writes
    kSiteBlockStage = 8,     // 2-D tile kernel: staged rows and quads
    kSiteBatchTile = 9,      // batch tile record within its member
    kSiteBatchBlockHeader = 10, // batch temporal blocking: a tile within its member, its rows within a plane
    kSiteBatchBlockStage = 11,  // ... the rows of a bulk copy within the staged plane
    kSiteBatchBlockQuad = 12,   // ... the rows and words a quad reads
    kSiteSelfTest = 99,      // fhp_debug_selftest
};

#ifdef FHP_DEBUG
constexpr bool kDebugBuild = true;
#else
constexpr bool kDebugBuild = false;
#endif

// True if `cond` holds; in the debug build a false `cond` is recorded in
// *err (if not NULL) and false returned, so that the caller skips the access.
__device__ __forceinline__ bool dbg_ok(bool cond, unsigned int* err, unsigned int site) {
#ifdef FHP_DEBUG
    if (!cond) {
        if (err) atomicOr(err, kErrBounds | (site << 8));
        return false;
    }
#endif
    (void)cond;
    (void)err;
    (void)site;
    return true;
}

// As dbg_ok, and the first failure of a launch also leaves `value` (16 bits)
// in bits 16..31 of the error word.
__device__ __forceinline__ bool dbg_ok_v(bool cond, unsigned int* err, unsigned int site, unsigned int value) {
#ifdef FHP_DEBUG
    if (!cond) {
        if (err) {
            const unsigned int word = kErrBounds | (site << 8) | ((value & 0xFFFFu) << 16);
            if (atomicCAS(err, 0u, word) != 0u) atomicOr(err, kErrBounds | (site << 8));
        }
        return false;
    }
#endif
    (void)cond;
    (void)err;
    (void)site;
    (void)value;
    return true;
}

}  // namespace fhp
