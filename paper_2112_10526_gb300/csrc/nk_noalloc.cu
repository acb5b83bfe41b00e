// nk_local_energy_noalloc: the local-energy entry point for callers that
// cannot let a library allocate device memory.
//
// Who needs it: programs whose device memory is owned by another allocator
// (a framework that reserves most of HBM up front, so a library cudaMalloc
// fails or fragments that pool), and latency-critical loops that cannot
// afford cudaMalloc / cudaFree, which synchronise the device and stall every
// other stream.  nk_local_energy keeps its tables in a context workspace
// that grows with cudaMalloc; this variant needs no context and keeps the
// same tables in one fixed array compiled into the library instead.
//
// The array is a file-scope __device__ variable of kNoallocScratchBytes.
// Every GPU that loads libnk.so holds it until the process exits.  Host code
// cannot use the array's name as a device address (in host code it names a
// host-side stand-in), so the device address is looked up with
// cudaGetSymbolAddress on the first call made with a device current, and
// cached per device together with the identity of the CUDA context it was
// looked up in.  A call made in another context on that device (after
// cudaDeviceReset, a primary-context reset, or with a driver-API context
// current) looks the address up again, since the module, and the array with
// it, may then live at another address.  Make the first call on a device,
// and the first call after such a reset, before any stream capture.
//
// All calls share the array and it keeps the last call's contents.  Every
// table a call reads is fully written by that same call first, so nothing
// has to start at zero.  Calls whose kernels overlap on the GPU (different
// streams, or different host threads) race on the array: serialise them.

#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/nk.h"
#include "nk_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[NK_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct ScratchSlot {
    unsigned long long ctx_id;  // identity of the context the address belongs to (0: none yet)
    char *addr;
};
ScratchSlot g_scratch_dev[kMaxDevices] = {};

// The driver's cuCtxGetCurrent / cuCtxGetId, reached through the runtime so
// that the library does not link libcuda directly.
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

// Identity of the context current on this thread (0 if none can be read).
unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != 0 || !ctx) return 0;
    if (get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of the scratch array in the context current on this thread
// (set-up on the first call per device and again whenever that context
// changes).
nk_status scratch_address(int dev, char **out) {
    if (dev < 0 || dev >= kMaxDevices) return nk::report_error(NK_ERR_INVALID_ARG, "device ordinal out of range");
    unsigned long long id = current_ctx_id();
    std::lock_guard<std::mutex> lk(g_mu);
    ScratchSlot &slot = g_scratch_dev[dev];
    if (id == 0 || slot.ctx_id != id || !slot.addr) {
        void *p = nullptr;
        // binds the device's primary context to this thread if none is current
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return nk::report_error(NK_ERR_CUDA, "cudaGetSymbolAddress(scratch) failed");
        }
        if (id == 0) id = current_ctx_id();
        slot.ctx_id = id;  // 0 (context identity unreadable): looked up again on every call
        slot.addr = static_cast<char *>(p);
    }
    *out = slot.addr;
    return NK_OK;
}

// A device (or managed) pointer that the kernels on device `dev` may use:
// memory of another GPU is rejected, since this entry point launches on the
// current device and peer access is not assumed.
bool on_device(const void *p, int dev) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Bump carving of the scratch array (base == nullptr counts bytes only).
struct Bump {
    char *base;
    size_t off = 0;
    template <class T>
    T *take(size_t n) {
        off = (off + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += n * sizeof(T);
        return p;
    }
};

template <typename R>
size_t plan_tables(Bump &b, nk::Tables<R> &t, const nk_rbm *rbm, const nk_ham *ham) {
    const int N = rbm->N, M = rbm->M, E = ham->n_edges;
    const bool site = ham->kind == NK_TFIM, edge = ham->kind == NK_HEIS;
    t.N = N;
    t.M = M;
    t.E = E;
    t.a = rbm->params;
    t.b = rbm->params + N;
    t.W = rbm->params + N + M;
    t.edges = ham->edges;
    t.Wt = b.take<double>((size_t)N * M);
    t.tau_site = site ? b.take<R>((size_t)N * M) : nullptr;
    t.tau_siteT = site ? b.take<R>((size_t)N * M) : nullptr;
    t.K_site = site ? b.take<R>(N) : nullptr;
    t.tau_edge = edge ? b.take<R>((size_t)E * M) : nullptr;
    t.tau_edgeT = edge ? b.take<R>((size_t)E * M) : nullptr;
    t.K_edge = edge ? b.take<R>(E) : nullptr;
    return b.off;
}

template <typename R>
nk_status run(int dev, const nk_rbm *rbm, const nk_ham *ham, const int8_t *s, int64_t Ns, double *eloc,
              double *t_out, cudaStream_t st) {
    nk::Tables<R> t{};
    Bump count{nullptr};
    const size_t need = plan_tables(count, t, rbm, ham);
    if (need > (size_t)NK_NOALLOC_SCRATCH_BYTES) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "nk_local_energy_noalloc: these sizes need %zu bytes of tables; the fixed scratch "
                 "holds %zu bytes (use nk_local_energy)",
                 need, (size_t)NK_NOALLOC_SCRATCH_BYTES);
        return nk::report_error(NK_ERR_INVALID_ARG, msg);
    }
    char *base = nullptr;
    nk_status stt = scratch_address(dev, &base);
    if (stt != NK_OK) return stt;
    Bump real{base};
    plan_tables(real, t, rbm, ham);
    const bool site = ham->kind == NK_TFIM, edge = ham->kind == NK_HEIS;
    cudaError_t e = nk::launch_tables(t, site, edge, st);
    if (e == cudaSuccess) {
        nk::ElocArgs a = nk::eloc_args(ham, s, Ns, eloc, t_out);
        e = nk::launch_eloc(t, a, st);
    }
    if (e != cudaSuccess) return nk::report_error(NK_ERR_CUDA, cudaGetErrorString(e));
    return NK_OK;
}

}  // namespace

extern "C" nk_status nk_local_energy_noalloc(const nk_rbm *rbm, int32_t precision, const nk_ham *ham,
                                             const int8_t *s, int64_t Ns, double *eloc_out,
                                             double *t_out, void *stream) {
    if (!rbm || !ham) return nk::report_error(NK_ERR_INVALID_ARG, "rbm or ham is NULL");
    if (rbm->N < 1 || rbm->N > 4096 || rbm->M < 1 || rbm->M > 8192)
        return nk::report_error(NK_ERR_INVALID_ARG, "N or M out of range");
    if (precision != NK_F64 && precision != NK_MIXED)
        return nk::report_error(NK_ERR_INVALID_ARG, "precision unknown");
    if (ham->kind != NK_TFIM && ham->kind != NK_HEIS)
        return nk::report_error(NK_ERR_INVALID_ARG, "ham->kind unknown");
    if (ham->n_edges < 1 || ham->n_edges > 65536)
        return nk::report_error(NK_ERR_INVALID_ARG, "ham->n_edges out of [1, 65536]");
    if (ham->n_edges2 < 0 || ham->n_edges2 > ham->n_edges)
        return nk::report_error(NK_ERR_INVALID_ARG, "ham->n_edges2 out of [0, n_edges]");
    if (Ns < 0) return nk::report_error(NK_ERR_INVALID_ARG, "Ns < 0");
    if (Ns == 0) return NK_OK;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return nk::report_error(NK_ERR_CUDA, cudaGetErrorString(e));
    if (!on_device(rbm->params, dev) || !on_device(ham->edges, dev) || !on_device(s, dev) ||
        !on_device(eloc_out, dev) || (t_out && !on_device(t_out, dev)))
        return nk::report_error(NK_ERR_INVALID_ARG,
                                "arrays must be device pointers of the current device");
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == NK_F64) return run<double>(dev, rbm, ham, s, Ns, eloc_out, t_out, st);
    return run<float>(dev, rbm, ham, s, Ns, eloc_out, t_out, st);
}
