// noalloc.cu -- qym_accel_dev_static: the E_Int acceleration of one system
// with its scratch in a fixed array inside the library instead of a
// caller-provided workspace, for callers that cannot allocate device memory.
#include <mutex>
#include <string>

#include "qym_internal.cuh"

namespace qym {

// Scratch of the static variant: float packs, heavy list, work items and
// partial sums for up to QYM_STATIC_MAX_ROWS rows (see accel_single_workspace).
// Every GPU that loads the library holds this array until the process exits.
constexpr size_t kStaticScratchBytes = (size_t)8 << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void *g_static_ptr[128];  // device address of the array, per device ordinal

// The array's name in host code is a host-side stand-in, not a device
// address. Its device address is looked up with the device current on every
// call that is not being captured into a CUDA graph (a lookup allocates
// nothing and is cheap), so a context torn down and created again (after
// cudaDeviceReset, say) gets the array's new address; during a capture the
// address from the last call on that device is used.
static cudaError_t static_scratch(cudaStream_t stream, void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = p;
    } else if (!g_static_ptr[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}

}  // namespace qym

static thread_local std::string g_static_err;

// errors go to the library's context-free message (qym_last_error(NULL)) and
// to this call's own getter, which returns the same text
static qym_status static_fail(qym_status st, const std::string &msg) {
    g_static_err = msg;
    qym::set_thread_error(msg);
    return st;
}

extern "C" const char *qym_static_last_error(void) { return g_static_err.c_str(); }

extern "C" size_t qym_static_scratch_bytes(void) { return qym::kStaticScratchBytes; }

extern "C" qym_status qym_accel_dev_static(int64_t rows, const double *m, const double *q,
                                           double *a, double G, int32_t prec, double heavy_mass,
                                           void *stream) {
    using namespace qym;
    if (rows < 2 || !m || !q || !a)
        return static_fail(QYM_EINVAL, "qym_accel_dev_static: rows < 2 or a NULL array");
    if (prec != QYM_KICK_FP64 && prec != QYM_KICK_MIXED)
        return static_fail(QYM_EINVAL,
                           "qym_accel_dev_static: prec must be QYM_KICK_FP64 or QYM_KICK_MIXED");
    if (rows > QYM_STATIC_MAX_ROWS)
        return static_fail(QYM_EINVAL, "qym_accel_dev_static: " + std::to_string(rows) +
                                           " rows exceed the fixed scratch limit of " +
                                           std::to_string((long long)QYM_STATIC_MAX_ROWS) +
                                           " rows; use qym_accel_dev with a caller workspace");
    size_t need = accel_single_workspace(rows, prec);
    if (need > kStaticScratchBytes)  // guarded by the row limit; checked anyway
        return static_fail(QYM_EINVAL, "qym_accel_dev_static: scratch of " +
                                           std::to_string(need) + " bytes exceeds the fixed array");
    void *scratch = nullptr;
    cudaError_t e = static_scratch((cudaStream_t)stream, &scratch);
    if (e == cudaSuccess)
        e = launch_accel_single(rows, m, q, a, G, prec, heavy_mass, scratch, kStaticScratchBytes,
                                (cudaStream_t)stream);
    if (e != cudaSuccess)
        return static_fail(QYM_ECUDA, std::string("qym_accel_dev_static: ") + cudaGetErrorString(e));
    return QYM_OK;
}
