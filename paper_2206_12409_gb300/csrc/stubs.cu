// Entry points whose implementation lives in later translation units are
// declared here until they exist.
#include "vsie_internal.h"
extern "C" {
vsie_status vsie_rhs_ports(vsie_ctx*, int32_t, const int32_t*, double, void*, int64_t, vsie_stream) {
    return VSIE_EUNSUPPORTED;
}
vsie_status vsie_solve(vsie_ctx*, int32_t, const void*, int64_t, void*, int64_t, double,
                       const vsie_solve_opts*, vsie_solve_info*, vsie_stream) {
    return VSIE_EUNSUPPORTED;
}
vsie_status vsie_save(const vsie_ctx*, const char*) { return VSIE_EUNSUPPORTED; }
vsie_status vsie_load(const char*, vsie_ctx** out) { if (out) *out = nullptr; return VSIE_EUNSUPPORTED; }
}
