// Entry points whose implementation lives in later translation units are
// declared here until they exist.
#include "vsie_internal.h"
extern "C" {
vsie_status vsie_save(const vsie_ctx*, const char*) { return VSIE_EUNSUPPORTED; }
vsie_status vsie_load(const char*, vsie_ctx** out) { if (out) *out = nullptr; return VSIE_EUNSUPPORTED; }
}
