// Body-operator matvec that allocates nothing (vsie_volume_matvec_static).
//
// Some callers cannot allocate device memory while they run this operator: a
// solver whose memory is owned by a fixed pool that must not grow, a real-time
// loop that may not block on the allocator, or a host runtime that hands out
// all device memory itself.  For them
// the two FFT work buffers of the fused convolution live in one file-scope
// device array of fixed size instead of in per-context allocations.  Every GPU
// that loads this library holds that array until the process exits.
#include "vsie_internal.h"

#include <mutex>

namespace vsie {

// Upper bound of the work buffers of one call (both FFT intermediates together).
constexpr size_t kStaticScratchBytes = 32ull << 20;   // 32 MiB

static __device__ __align__(256) unsigned char g_conv_scratch[kStaticScratchBytes];

// Device address of g_conv_scratch per device, looked up once per device with
// that device current.  In host code the symbol is only a stand-in for the
// device array, so kernels must be given this address, never the symbol.
static std::mutex g_scratch_mu;
static void* g_scratch_addr[64] = {nullptr};

static void* scratch_address() {
    int dev = 0;
    VSIE_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) throw Error(VSIE_EUNSUPPORTED, "device index above 63");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_conv_scratch);
        if (e != cudaSuccess)
            throw Error(VSIE_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    return g_scratch_addr[dev];
}

template <typename R>
void conv_apply_given_scratch(Ctx& c, int p, const cx<R>* Xb, int64_t ldx, cx<R>* Yb, int64_t ldy,
                              cx<R>* A, cx<R>* B, cudaStream_t st);

template <typename R>
static vsie_status run(Ctx& c, int p, const void* Xb, int64_t ldx, void* Yb, int64_t ldy,
                       cudaStream_t st) {
    const size_t cs = sizeof(cx<R>);
    const size_t nA = (size_t)p * 3 * c.ne[2] * c.ne[1] * c.L[0];
    const size_t nB = (size_t)p * 3 * c.ne[2] * c.L[1] * c.L[0];
    const size_t offB = (nA * cs + 255) / 256 * 256;
    if (offB + nB * cs > kStaticScratchBytes)
        throw Error(VSIE_EINVAL, "grid and p need " + std::to_string(offB + nB * cs) +
                                     " bytes of work space; the static limit is " +
                                     std::to_string(kStaticScratchBytes));
    unsigned char* base = (unsigned char*)scratch_address();
    conv_apply_given_scratch<R>(c, p, (const cx<R>*)Xb, ldx, (cx<R>*)Yb, ldy, (cx<R>*)base,
                                (cx<R>*)(base + offB), st);
    return VSIE_OK;
}

}  // namespace vsie

using namespace vsie;

extern "C" vsie_status vsie_volume_matvec_static(vsie_ctx* ctx, int32_t p, const void* Xb,
                                                 int64_t ldx, void* Yb, int64_t ldy,
                                                 int32_t precision, vsie_stream stream) {
    if (!ctx) { set_global_err("null context"); return VSIE_EINVAL; }
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    try {
        if (!Xb || !Yb) throw Error(VSIE_EINVAL, "null X or Y");
        if (p < 1) throw Error(VSIE_EINVAL, "p must be >= 1");
        if (ldx < 3 * c->n_b || ldy < 3 * c->n_b) throw Error(VSIE_EINVAL, "leading dimension < 3 n_b");
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        if (precision == VSIE_C128) {
            if (!c->f64.ready) throw Error(VSIE_EUNSUPPORTED, "context built without C128");
            return run<double>(*c, p, Xb, ldx, Yb, ldy, st);
        }
        if (precision == VSIE_C64) {
            if (!c->f32.ready) throw Error(VSIE_EUNSUPPORTED, "context built without C64");
            return run<float>(*c, p, Xb, ldx, Yb, ldy, st);
        }
        throw Error(VSIE_EINVAL, "unknown precision");
    } catch (const Error& e) {
        c->err = e.msg;
        return e.st;
    }
}
