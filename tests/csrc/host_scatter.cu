// Test-only: the device scattering expressions of the CUDA library, compiled
// for the host, so that the not-gpu tests can compare them with the oracle's
// 256-entry tables over every node state.  Not part of the product library.
#include <cstdint>

#include "../../paper_1208_2428_gb300/csrc/fhp_device.cuh"

extern "C" __attribute__((visibility("default"))) void host_scatter_words(
    const uint32_t* planes7, uint32_t solid, uint32_t chi, uint32_t rest_rules, uint32_t* out7) {
    fhp::Planes7 in{planes7[0], planes7[1], planes7[2], planes7[3], planes7[4], planes7[5], planes7[6]};
    const fhp::Planes7 o = fhp::scatter(in, solid, chi, rest_rules);
    out7[0] = o.m0; out7[1] = o.m1; out7[2] = o.m2; out7[3] = o.m3;
    out7[4] = o.m4; out7[5] = o.m5; out7[6] = o.rest;
}

extern "C" __attribute__((visibility("default"))) void host_scatter_saturated_words(
    const uint32_t* planes7, uint32_t solid, uint32_t chi, uint32_t* out7) {
    fhp::Planes7 in{planes7[0], planes7[1], planes7[2], planes7[3], planes7[4], planes7[5], planes7[6]};
    const fhp::Planes7 o = fhp::scatter_saturated(in, solid, chi);
    out7[0] = o.m0; out7[1] = o.m1; out7[2] = o.m2; out7[3] = o.m3;
    out7[4] = o.m4; out7[5] = o.m5; out7[6] = o.rest;
}
