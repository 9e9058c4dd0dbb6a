// fhp_static.cu -- fhp_run_static: an FHP run that allocates no device memory.
//
// Some callers cannot allocate device memory: plugins whose host application
// owns all GPU memory through its own pool, services that fix a hard memory
// cap at start-up, and latency-critical loops where an allocation (which may
// synchronise the device) is not acceptable.  This entry point serves them:
// the caller passes device buffers for the input and output node bytes, and
// every intermediate buffer (the two bit-plane state buffers, the solid plane
// and a flag word) lives in one file-scope __device__ array of fixed size.
//
// That array exists once per GPU that loads the library and stays allocated
// until the process exits.  All calls on a device share it and it keeps the
// previous call's contents, so calls whose work overlaps on the GPU (from two
// streams or two host threads) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/fhp.h"
#include "fhp_internal.h"

namespace {

constexpr size_t kScratchBytes = FHP_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};   // context the address belongs to

size_t round256(size_t v) { return (v + 255) / 256 * 256; }

// Identity of the calling thread's current CUDA context (0 if none or if the
// driver cannot say), from the driver's cuCtxGetCurrent and cuCtxGetId looked
// up through the runtime (no link against the driver library).
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);

unsigned long long current_context_id() {
    static std::once_flag once;
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)f;
        cudaGetLastError();
    });
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of the scratch array on the current device.  Set-up, once
// per device (with that device current): cudaGetSymbolAddress, which needs no
// allocation, its result checked and kept.  A later call reuses it while the
// device's context is the same one; after the context was destroyed and made
// again (cudaDeviceReset) the module may sit elsewhere, so the address is
// looked up again.  If the context's identity cannot be read, every call
// looks the address up.
cudaError_t scratch_address(int device, void** out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_addr[device] || ctx == 0 || ctx != g_scratch_ctx[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = p;
        // The look-up initialises the context if it did not exist yet.
        g_scratch_ctx[device] = ctx ? ctx : current_context_id();
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

int fail(int code, const char* msg) {
    fhp::set_thread_error(msg);  // reported by fhp_last_error(NULL)
    return code;
}

}  // namespace

extern "C" FHP_API int fhp_run_static(const uint8_t* device_bytes_in, uint8_t* device_bytes_out,
                                      int32_t width, int32_t height, uint64_t seed, int64_t t0,
                                      int64_t n, double forcing_p, void* stream) {
    if (!device_bytes_in || !device_bytes_out) return fail(FHP_EINVAL, "fhp_run_static: NULL buffer");
    if (width < 32 || width % 32 != 0 || height < 2 || height % 2 != 0)
        return fail(FHP_EINVAL, "fhp_run_static: W must be a positive multiple of 32 and H even >= 2");
    if (n < 0 || t0 < 0 || t0 > ((int64_t)1 << 48) - n)
        return fail(FHP_EINVAL, "fhp_run_static: need n >= 0 and 0 <= t0, t0 + n < 2^48");
    if (!(forcing_p >= 0.0 && forcing_p <= 1.0))
        return fail(FHP_EINVAL, "fhp_run_static: forcing probability outside [0, 1]");
    const fhp::Geometry g = fhp::make_geometry(width, height);
    const size_t plane_bytes = round256(g.plane_words * sizeof(uint32_t));
    const size_t need = 15 * plane_bytes + 256;
    if (need > kScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "fhp_run_static: a %d x %d lattice needs %zu bytes of scratch; the static scratch holds %zu",
                 width, height, need, kScratchBytes);
        return fail(FHP_EINVAL, msg);
    }
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess || device < 0 || device >= kMaxDevices)
        return fail(FHP_ECUDA, "fhp_run_static: no usable current device");
    void* base = nullptr;
    e = scratch_address(device, &base);
    if (e != cudaSuccess) return fail(FHP_ECUDA, "fhp_run_static: cudaGetSymbolAddress failed");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* b = (unsigned char*)base;
    uint32_t* buf[2] = {(uint32_t*)b, (uint32_t*)(b + 7 * plane_bytes)};
    uint32_t* solid = (uint32_t*)(b + 14 * plane_bytes);
    unsigned int* flag = (unsigned int*)(b + 15 * plane_bytes);
    // The pack kernel writes every word of every plane (padding included);
    // only the flag word has to start at zero.
    e = cudaMemsetAsync(flag, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) e = fhp::launch_pack(g, device_bytes_in, buf[0], solid, flag, s);
    const fhp::ForcingTable ft = fhp::forcing_table(forcing_p);
    const bool force = ft.q[32] != 0;
    const fhp::Key2 key{(uint32_t)seed, (uint32_t)(seed >> 32)};
    int cur = 0;
    for (int64_t i = 0; i < n && e == cudaSuccess; ++i) {
        // The solid plane is always read (it is all zero when there are no
        // obstacles), so no host read-back of the solid flag is needed.  The
        // direct kernel is used because it has no device-side waits: the
        // call is asynchronous and could not report a wait that gave up.
        e = fhp::launch_step(g, buf[cur], buf[cur ^ 1], solid, true, force, ft, key, (uint64_t)(t0 + i), s,
                             nullptr, fhp::kStepDirect);
        cur ^= 1;
    }
    if (e == cudaSuccess) e = fhp::launch_unpack(g, buf[cur], solid, device_bytes_out, s);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "fhp_run_static: %s", cudaGetErrorString(e));
        return fail(FHP_ECUDA, msg);
    }
    return FHP_OK;
}
