// chem_api.cu -- C ABI entry points for the source term: argument checks and dispatch.
#include "chem_internal.h"

using namespace chem;

namespace chem {
int *bf16_status_word(const chem_mech *m);
chem_status launch_source_bf16(const chem_mech *m, int64_t n, const float *T, const float *P,
                               const float *Y, int64_t ldY, float *om, int64_t ldO,
                               cudaStream_t s);
}

static chem_status check_device(const chem_mech *m)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(CHEM_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev != m->device)
        return set_error(CHEM_EINVAL, "mechanism lives on device %d, current device is %d",
                         m->device, dev);
    return CHEM_OK;
}

extern "C" chem_status chem_source_term(const chem_mech *m, int64_t n, const void *T,
                                        const void *P, const void *Y, int64_t ldY, void *om,
                                        int64_t ldO, chem_precision prec, void *stream)
{
    clear_error();
    if (!m) return set_error(CHEM_EINVAL, "mechanism is NULL");
    if (n < 0) return set_error(CHEM_EINVAL, "n_cells < 0");
    if (ldY < m->ns || ldO < m->ns)
        return set_error(CHEM_EINVAL, "ldY=%lld / ldO=%lld below n_species=%d", (long long)ldY,
                         (long long)ldO, m->ns);
    if (prec != CHEM_FP64 && prec != CHEM_FP32 && prec != CHEM_SPLIT_BF16)
        return set_error(CHEM_EINVAL, "unknown precision %d", (int)prec);
    if (n == 0) return CHEM_OK;
    if (!T || !P || !Y || !om) return set_error(CHEM_EINVAL, "NULL array with n_cells > 0");
    chem_status st = check_device(m);
    if (st != CHEM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    switch (prec) {
    case CHEM_FP64:
        return launch_source_fp64(m, n, (const double *)T, (const double *)P, (const double *)Y,
                                  ldY, (double *)om, ldO, s);
    case CHEM_FP32:
        return launch_source_fp32(m, n, (const float *)T, (const float *)P, (const float *)Y, ldY,
                                  (float *)om, ldO, s);
    default:
        return launch_source_bf16(m, n, (const float *)T, (const float *)P, (const float *)Y, ldY,
                                  (float *)om, ldO, s);
    }
}

// ---------------------------------------------------------------------------------------
// host-buffer entry: chunked H2D -> kernel -> D2H on three library-owned streams
// ---------------------------------------------------------------------------------------

#include <mutex>

namespace {

constexpr int kPipe = 3;         // stages: H2D of chunk i + 2, kernel of i + 1, D2H of i

struct HostPipe {
    cudaStream_t st[kPipe] = {};
    cudaEvent_t ev_in = nullptr, ev_out[kPipe] = {};
    bool ok = false;
};

HostPipe g_pipes[64];
std::mutex g_pipe_mu;

chem_status get_pipe(int dev, HostPipe **out)
{
    if (dev < 0 || dev >= 64) return set_error(CHEM_EUNSUPPORTED, "device index %d", dev);
    std::lock_guard<std::mutex> g(g_pipe_mu);
    HostPipe &p = g_pipes[dev];
    if (!p.ok) {
        for (int i = 0; i < kPipe; ++i) {
            if (cudaStreamCreateWithFlags(&p.st[i], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&p.ev_out[i], cudaEventDisableTiming) != cudaSuccess)
                return set_error(CHEM_ECUDA, "stream/event creation failed");
        }
        if (cudaEventCreateWithFlags(&p.ev_in, cudaEventDisableTiming) != cudaSuccess)
            return set_error(CHEM_ECUDA, "event creation failed");
        p.ok = true;
    }
    *out = &p;
    return CHEM_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t stage_bytes(int ns, int64_t chunk, int64_t ldY, size_t elt)
{
    return align256(elt * chunk) * 2 + align256(elt * chunk * ldY) + align256(elt * chunk * ns);
}

}  // namespace

extern "C" size_t chem_source_term_host_workspace(const chem_mech *m, int64_t chunk,
                                                  int64_t ldY, chem_precision prec)
{
    if (!m || chunk < 1 || ldY < 1) return 0;
    size_t elt = prec == CHEM_FP64 ? 8 : 4;
    return kPipe * stage_bytes(m->ns, chunk, ldY, elt);
}

extern "C" chem_status chem_source_term_host(const chem_mech *m, int64_t n, const void *T,
                                             const void *P, const void *Y, int64_t ldY,
                                             void *om, int64_t ldO, chem_precision prec,
                                             int64_t chunk, void *ws, size_t ws_bytes,
                                             void *stream)
{
    clear_error();
    if (!m) return set_error(CHEM_EINVAL, "mechanism is NULL");
    if (n < 0) return set_error(CHEM_EINVAL, "n_cells < 0");
    if (ldY < m->ns || ldO < m->ns)
        return set_error(CHEM_EINVAL, "ldY / ldO below n_species=%d", m->ns);
    if (prec != CHEM_FP64 && prec != CHEM_FP32 && prec != CHEM_SPLIT_BF16)
        return set_error(CHEM_EINVAL, "unknown precision %d", (int)prec);
    if (chunk < 1) return set_error(CHEM_EINVAL, "chunk_cells < 1");
    if (n == 0) return CHEM_OK;
    if (!T || !P || !Y || !om) return set_error(CHEM_EINVAL, "NULL array with n_cells > 0");
    if (!ws || ((uintptr_t)ws & 255))
        return set_error(CHEM_EINVAL, "workspace must be non-NULL and 256-byte aligned");
    if (chunk > n) chunk = n;
    const size_t need = chem_source_term_host_workspace(m, chunk, ldY, prec);
    if (ws_bytes < need)
        return set_error(CHEM_EINVAL, "workspace of %zu bytes below the %zu needed", ws_bytes,
                         need);
    chem_status st = check_device(m);
    if (st != CHEM_OK) return st;
    HostPipe *pp = nullptr;
    if ((st = get_pipe(m->device, &pp)) != CHEM_OK) return st;
    const size_t elt = prec == CHEM_FP64 ? 8 : 4;
    const int ns = m->ns;
    cudaStream_t user = (cudaStream_t)stream;
    cudaError_t e = cudaEventRecord(pp->ev_in, user);
    for (int i = 0; i < kPipe && e == cudaSuccess; ++i)
        e = cudaStreamWaitEvent(pp->st[i], pp->ev_in, 0);
    const size_t sb = stage_bytes(ns, chunk, ldY, elt);
    int64_t c = 0;
    for (int64_t lo = 0; lo < n && e == cudaSuccess; lo += chunk, ++c) {
        const int64_t cnt = (n - lo < chunk) ? n - lo : chunk;
        const int b = (int)(c % kPipe);
        cudaStream_t s = pp->st[b];
        unsigned char *base = (unsigned char *)ws + sb * b;
        void *dT = base;
        void *dP = base + align256(elt * chunk);
        void *dY = base + 2 * align256(elt * chunk);
        void *dO = base + 2 * align256(elt * chunk) + align256(elt * chunk * ldY);
        e = cudaMemcpyAsync(dT, (const char *)T + lo * elt, cnt * elt, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dP, (const char *)P + lo * elt, cnt * elt, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dY, (const char *)Y + lo * ldY * elt, cnt * ldY * elt,
                                cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) break;
        switch (prec) {
        case CHEM_FP64:
            st = launch_source_fp64(m, cnt, (const double *)dT, (const double *)dP,
                                    (const double *)dY, ldY, (double *)dO, ns, s);
            break;
        case CHEM_FP32:
            st = launch_source_fp32(m, cnt, (const float *)dT, (const float *)dP,
                                    (const float *)dY, ldY, (float *)dO, ns, s);
            break;
        default:
            st = launch_source_bf16(m, cnt, (const float *)dT, (const float *)dP,
                                    (const float *)dY, ldY, (float *)dO, ns, s);
        }
        if (st != CHEM_OK) break;
        // contiguous rows (ldO == n_species): one linear copy; a pitched copy of narrow rows
        // moves far fewer bytes per second
        if (ldO == ns)
            e = cudaMemcpyAsync((char *)om + lo * ldO * elt, dO, cnt * ns * elt,
                                cudaMemcpyDeviceToHost, s);
        else
            e = cudaMemcpy2DAsync((char *)om + lo * ldO * elt, ldO * elt, dO, ns * elt, ns * elt,
                                  cnt, cudaMemcpyDeviceToHost, s);
    }
    // the caller's stream waits for both pipeline streams, even after an error
    for (int i = 0; i < kPipe; ++i) {
        cudaEventRecord(pp->ev_out[i], pp->st[i]);
        cudaStreamWaitEvent(user, pp->ev_out[i], 0);
    }
    if (st != CHEM_OK) return st;
    if (e != cudaSuccess) return set_error(CHEM_ECUDA, "host pipeline: %s", cudaGetErrorString(e));
    return CHEM_OK;
}

extern "C" chem_status chem_device_status(const chem_mech *m, int32_t *code)
{
    clear_error();
    if (!m || !code) return set_error(CHEM_EINVAL, "NULL argument");
    *code = 0;
    chem_status st = check_device(m);
    if (st != CHEM_OK) return st;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return set_error(CHEM_ECUDA, "synchronize: %s", cudaGetErrorString(e));
    int *w = bf16_status_word(m);
    if (!w) return CHEM_OK;
    int v = 0;
    e = cudaMemcpy(&v, w, sizeof v, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && v != 0) e = cudaMemset(w, 0, sizeof v);
    if (e != cudaSuccess) return set_error(CHEM_ECUDA, "status word: %s", cudaGetErrorString(e));
    *code = v;
    return CHEM_OK;
}
