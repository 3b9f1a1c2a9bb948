// awpm_search_noalloc: the cycle search (Steps A-C) for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: a host framework that has already
// handed the whole GPU to its own memory pool, or code running where an
// allocation (which may synchronise the device) is not allowed.  This entry
// point therefore allocates nothing.  Its scratch lives in one file-scope
// __device__ array of fixed size (kScratchBytes, about 19 MB), which every
// GPU that loads the library keeps until the process exits.  The caller
// passes every input and output in device memory.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "awpm.h"
#include "awpm_internal.h"

using namespace awpm;

namespace {

constexpr int32_t kMaxN = AWPM_NOALLOC_MAX_N;
constexpr int32_t kMaxNnz = AWPM_NOALLOC_MAX_NNZ;
constexpr size_t kAlign = 256;

constexpr size_t up(size_t x)
{
    return (x + kAlign - 1) / kAlign * kAlign;
}

// Layout of the scratch array (byte offsets, each 256-byte aligned).
constexpr size_t kTilesMax = ((size_t)kMaxNnz + kTile - 1) / kTile + 1;
constexpr size_t kOffWork = 0;
constexpr size_t kOffCtl = kOffWork + up(sizeof(Work));
constexpr size_t kOffMc = kOffCtl + up(sizeof(Ctl));
constexpr size_t kOffMr = kOffMc + up(sizeof(int32_t) * kMaxN);
constexpr size_t kOffWm = kOffMr + up(sizeof(int32_t) * kMaxN);
constexpr size_t kOffRr = kOffWm + up(sizeof(double) * kMaxN);
constexpr size_t kOffRsig = kOffRr + up(sizeof(RowRange) * kMaxN);
constexpr size_t kOffSig = kOffRsig + up(sizeof(unsigned long long) * kMaxN);
constexpr size_t kOffBest = kOffSig + up(sizeof(unsigned long long) * kMaxN);
constexpr size_t kOffWin = kOffBest + up(sizeof(Rec) * kMaxN);
constexpr size_t kOffWkey = kOffWin + up(sizeof(uint32_t) * (kMaxN / 32 + 1));
constexpr size_t kOffTile = kOffWkey + up(sizeof(int32_t) * kMaxN);
constexpr size_t kOffStarts = kOffTile + up(sizeof(int32_t) * kTilesMax);
constexpr size_t kOffWpart = kOffStarts + up(sizeof(uint32_t) * (kMaxNnz / 32 + 1));
constexpr size_t kScratchBytes = kOffWpart + up(sizeof(double) * kWsumBlocks);

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch on the current device.  In host code the name
// g_scratch is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress with the device current.  It is looked up on every
// call (a table lookup once the module is loaded), so a context re-created
// after cudaDeviceReset never sees a stale address.
int scratch_address(unsigned char **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return AWPM_ERR_CUDA;
    }
    *out = (unsigned char *)p;
    return AWPM_OK;
}

bool on_device(const void *p, int device)
{
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == device) ||
           a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int awpm_search_noalloc(int32_t n, const int32_t *colptr, const int32_t *rowidx,
                                   const double *weight, const int32_t *mate, double *stepc_gain,
                                   int32_t *stepc_row, void *stream, awpm_stats *stats)
{
    if (n < 0)
        return AWPM_ERR_INVALID_ARG;
    if (n > kMaxN)
        return AWPM_ERR_TOO_LARGE;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return AWPM_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    awpm_stats S;
    std::memset(&S, 0, sizeof(S));
    S.lookup_used = AWPM_LOOKUP_BSEARCH;
    if (n == 0) {
        S.converged = 1;
        if (stats)
            *stats = S;
        return AWPM_OK;
    }
    if (!on_device(colptr, device) || !on_device(mate, device) ||
        !on_device(stepc_gain, device) || !on_device(stepc_row, device))
        return AWPM_ERR_INVALID_ARG;
    int32_t nnz = 0;
    if (cudaMemcpyAsync(&nnz, colptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return AWPM_ERR_CUDA;
    }
    if (nnz < 0 || (nnz > 0 && (!on_device(rowidx, device) || !on_device(weight, device))))
        return AWPM_ERR_INVALID_ARG;
    if (nnz > kMaxNnz)
        return AWPM_ERR_TOO_LARGE;

    unsigned char *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != AWPM_OK)
        return rc;
    int num_sms = 1;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return AWPM_ERR_CUDA;
    }

    Work wk;
    std::memset(&wk, 0, sizeof(wk));
    wk.n = n;
    wk.nnz = nnz;
    wk.ntiles = (int32_t)(((int64_t)nnz + kTile - 1) / kTile);
    wk.max_passes = 1;
    wk.lookup = AWPM_LOOKUP_BSEARCH;
    wk.htab = nullptr;
    wk.colptr = colptr;
    wk.rowidx = rowidx;
    wk.w = weight;
    wk.mate_in = mate;
    wk.ctl = (Ctl *)(base + kOffCtl);
    wk.mc = (int32_t *)(base + kOffMc);
    wk.mr = (int32_t *)(base + kOffMr);
    wk.wm = (double *)(base + kOffWm);
    wk.rrange = (RowRange *)(base + kOffRr);
    wk.rsig = (unsigned long long *)(base + kOffRsig);
    wk.colsig = (unsigned long long *)(base + kOffSig);
    wk.best = (Rec *)(base + kOffBest);
    // the search never selects (Step D): its selection records share the
    // Step-C area, which launch_init clears either way
    wk.dsel = (Sel *)(base + kOffBest);
    wk.winbits = (uint32_t *)(base + kOffWin);
    wk.wkey = (int32_t *)(base + kOffWkey);
    wk.tile_col = (int32_t *)(base + kOffTile);
    wk.starts = (uint32_t *)(base + kOffStarts);
    wk.wpart = (double *)(base + kOffWpart);

    // launch_init clears everything that must start at zero (control block,
    // row mates, column-start bits, column signatures, Step-C and Step-D
    // records) before use.
    // the descriptor lives in the scratch array too; the kernels read it there
    Work *d = (Work *)(base + kOffWork);
    if (cudaMemcpyAsync(d, &wk, sizeof(Work), cudaMemcpyHostToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return AWPM_ERR_CUDA;
    }
    Shape sh;
    sh.num_sms = num_sms;
    sh.wide = default_search_wide();
    sh.search_bps = search_blocks_per_sm(AWPM_LOOKUP_BSEARCH, false, sh.wide);
    sh.lookup = AWPM_LOOKUP_BSEARCH;
    sh.batch = false;
    sh.search_waves = search_waves(num_sms, sh.search_bps, wk.ntiles);
    Sink k;
    k.stream = s;
    launch_init(d, sh, k);
    launch_search(d, sh, k);
    launch_export_stepc(d, sh, stepc_gain, stepc_row, k);
    if (k.err != cudaSuccess) {
        cudaGetLastError();
        return AWPM_ERR_CUDA;
    }
    Ctl h;
    if (cudaMemcpyAsync(&h, wk.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return AWPM_ERR_CUDA;
    }
    if (h.err)
        return awpm_code_of_bits(h.err);
    S.iterations = 0;
    S.converged = 0;
    S.edge_checks = (int64_t)nnz - n;
    S.candidates = (int64_t)h.candidates;
    S.closing_found = (int64_t)h.found;
    S.positive = (int64_t)h.positive;
    if (stats)
        *stats = S;
    return AWPM_OK;
}
