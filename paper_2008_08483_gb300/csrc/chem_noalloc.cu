// chem_noalloc.cu -- chem_integrate_cells_noalloc: the reactor integration of
// chem_integrate_cells with its device workspace taken from a fixed static array instead of
// a per-call allocation.
//
// Why: chem_integrate_cells allocates its workspace (the cell queue and failure count, plus
// per-warp matrices for mechanisms too large for shared memory) on the caller's stream.
// Some callers cannot allow that: a CFD solver or framework that has handed all device
// memory to its own pool allocator, where an allocation by the library would fail or
// fragment that pool, and time-step loops that must not pay an allocation's latency or
// its possible implicit synchronisation.  This entry point allocates nothing: no
// cudaMalloc / cudaMallocAsync / cudaFree, no allocating library routine.
//
// The workspace is kNoAllocScratchBytes (1 MiB) of static device memory per device, shared
// by every call on that device.  The part that must start at zero (the 256-byte header:
// next-cell counter and failure count) is cleared on the stream by each call before its
// kernel runs; nothing else needs initialising.  Calls that overlap in time on the same
// device (different streams or host threads) race on this array and must not be issued.
// Mechanisms whose reactor matrices do not fit in shared memory need per-warp matrices in
// device memory, which this entry point does not provide: they are rejected (CHEM_ENOMEM)
// whatever the cell count, so the limit is a property of the mechanism alone.
// Each call looks up the array's address with cudaGetSymbolAddress (which allocates
// nothing) with the current device; a device reset therefore never leaves a stale address
// behind.  The first call on a device may load the module that holds the array; make it
// before any stream capture on that device.
#include "chem_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = 1u << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Address of the scratch array on the current device, looked up on every call.
chem_status scratch_for_current_device(void **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return chem::set_error(CHEM_ECUDA, "cudaGetSymbolAddress of the static scratch: %s",
                               cudaGetErrorString(e));
    *out = p;
    return CHEM_OK;
}

}  // namespace

using namespace chem;

extern "C" chem_status chem_integrate_cells_noalloc(const chem_mech *m, int64_t n, double *T,
                                                    const double *P, double *Y, int64_t ldY,
                                                    double t_end, double rtol, double atol,
                                                    const chem_integrate_opts *opts,
                                                    int32_t *cell_status, void *stream)
{
    clear_error();
    chem_status st = integrate_checks(m, n, T, P, Y, ldY, t_end, rtol, atol);
    if (st != CHEM_OK) return st;
    if (n == 0) return CHEM_OK;
    // per-warp reactor matrices in device memory (mechanisms beyond shared memory) are not
    // provided, whatever n is; the rest of the workspace is the fixed header
    const size_t need = integrate_workspace_bytes(m, 1);
    if (need > integrate_header_bytes() || need > kNoAllocScratchBytes)
        return set_error(CHEM_ENOMEM,
                         "integrate (no allocation): the mechanism's reactor matrices exceed "
                         "shared memory and would need %zu bytes per cell-group of workspace "
                         "beyond the static scratch's header",
                         need - integrate_header_bytes());
    void *ws = nullptr;
    st = scratch_for_current_device(&ws);
    if (st != CHEM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = integrate_launch(m, n, nullptr, T, P, Y, ldY, t_end, rtol, atol, opts, cell_status, ws,
                          kNoAllocScratchBytes, s);
    if (st != CHEM_OK) return st;
    unsigned int h_fail = 0;
    cudaError_t e = cudaMemcpyAsync(&h_fail, (unsigned int *)ws + 1, sizeof h_fail,
                                    cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return set_error(CHEM_ECUDA, "integrate (no allocation): %s", cudaGetErrorString(e));
    if (h_fail)
        return set_error(CHEM_ENONCONV, "integrate: %u of %lld cells failed", h_fail, (long long)n);
    return CHEM_OK;
}
