// bx_noalloc.cu -- the forward response stage for callers that cannot allocate device memory.
//
// Who needs this: code that must not call cudaMalloc on the hot path -- a host process whose
// device memory is owned by another allocator (a framework's caching pool or a budget fixed at
// start-up), a loop where cudaMalloc's implicit device synchronisation would stall work on
// other streams, or an embedded/real-time host that forbids allocation after initialisation.
// Such a caller owns its input and output buffers and wants the library to add nothing.
//
// bx_spectra_noalloc runs the per-column stage and the FP32 rate-first forward kernel (the
// same kernels as bx_nll_batch) for one dataset at one parameter point.  Their scratch (the
// per-column parameters, band limits, the dataset descriptor, status words) lives in the
// file-scope device array g_noalloc_scratch of fixed size: nothing is allocated, ever.
//
// Consequences for the caller:
//   * the array's device address is looked up once per device, on the first call made with
//     that device current;
//   * every call on a device shares the one array, so calls that overlap on the GPU (two
//     streams, two host threads) race: serialise them;
//   * the array keeps whatever the last call left in it; each call re-initialises everything
//     it reads: the dataset descriptor arrives as a kernel argument (copied at launch, so the
//     call never waits on a host-to-device copy from pageable memory), and the status words
//     are rewritten before the stages run;
//   * a parameter point outside the model's domain (non-finite theta, LY <= 0, sigma^2 <= 0)
//     fills lambda with NaN, so stale contents of the caller's buffer are never mistaken for
//     spectra.
#include <cuda_runtime.h>

#include <mutex>

#include "bx_internal.cuh"
#include "bx_model.h"

using namespace bx;

namespace {

constexpr int NA_MAX_GRID = 4096;   // true-energy points
constexpr int NA_MAX_ROWS = 4096;   // output bins
constexpr int NA_MAX_DEVICES = 64;

struct NoAllocScratch {
    Toy toy;
    int toy_of;
    int status;
    unsigned err;
    unsigned pad;
    unsigned long long units;
    Col64 col64[NA_MAX_GRID];
    double2 colq[NA_MAX_GRID];
    float4 colf[NA_MAX_GRID];
    ColG colg[NA_MAX_GRID];
    double2 colS[NA_MAX_GRID];
    float4 colS32[NA_MAX_GRID];
    float colAl[NA_MAX_GRID];
    double aW[NA_MAX_GRID];
    int2 colr[NA_MAX_GRID];
    int2 tile_cols[MAX_TILES];
    int2 cb_rows[MAX_CB];
};

std::mutex g_lookup_mutex;
void* g_scratch_addr[NA_MAX_DEVICES] = {};

}  // namespace

// 530 KiB per device that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

// Store the dataset descriptor (passed by value) and clear the status words of the scratch.
__global__ void k_noalloc_begin(Toy t, NoAllocScratch* scr) {
    scr->toy = t;
    scr->toy_of = 0;
    scr->status = 0;
    scr->err = 0u;
}

// After the forward: when the column stage rejected the parameter point, lambda is NaN.
__global__ void k_noalloc_end(const NoAllocScratch* scr, double* lambda, int n) {
    if (scr->status == 0) return;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) lambda[j] = nan;
}

static int noalloc_scratch(NoAllocScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bx_set_error(BX_ECUDA, "bx_spectra_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return bx_set_error(BX_EINVAL, "bx_spectra_noalloc: device %d not supported", dev);
    std::lock_guard<std::mutex> lock(g_lookup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return bx_set_error(BX_ECUDA, "bx_spectra_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<NoAllocScratch*>(g_scratch_addr[dev]);
    return BX_OK;
}

extern "C" int bx_spectra_noalloc(int n_grid, double e_max, int n_species, const double* shapes,
                                  const double* stop_pow, const double* tag_frac, double width, int m_hi,
                                  const double* theta, double* lambda, void* cuda_stream) {
    if (n_grid < 1 || n_grid > NA_MAX_GRID)
        return bx_set_error(BX_EINVAL, "bx_spectra_noalloc: n_grid %d out of [1, %d] (fixed scratch size)", n_grid,
                            NA_MAX_GRID);
    if (m_hi < 1 || m_hi > NA_MAX_ROWS)
        return bx_set_error(BX_EINVAL, "bx_spectra_noalloc: m_hi %d out of [1, %d] (fixed scratch size)", m_hi,
                            NA_MAX_ROWS);
    if (n_species < 1 || n_species > KMAX)
        return bx_set_error(BX_EINVAL, "bx_spectra_noalloc: n_species %d out of [1, %d]", n_species, KMAX);
    if (!(e_max > 0.0) || !(width > 0.0))
        return bx_set_error(BX_EINVAL, "bx_spectra_noalloc: e_max and width must be > 0");
    if (!shapes || !stop_pow || !theta || !lambda)
        return bx_set_error(BX_EINVAL, "bx_spectra_noalloc: NULL device pointer");
    NoAllocScratch* scr = nullptr;
    int st = noalloc_scratch(&scr);
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    Toy T{};
    T.K = n_species;
    T.N = n_grid;
    T.n_set = 1;
    T.Ncs = T.Next = n_grid;
    T.set_of[0] = 0;
    T.xi[0] = 1.0;
    T.M = m_hi;
    T.m_lo = 0;
    T.nw = m_hi;
    T.n_es = 1;   // one energy slice: the whole axis
    T.es_lo[0] = 0;
    T.es_hi[0] = m_hi;
    T.L = 1;
    T.has_tag = tag_frac ? 1 : 0;
    T.nb = m_hi * (1 + T.has_tag);
    T.P = n_species + 7;
    T.n_tiles = (m_hi + TM - 1) / TM;
    T.n_cb = (n_grid + BCOLS - 1) / BCOLS;
    T.n_kb = (n_grid + KB - 1) / KB;
    T.dE = e_max / n_grid;
    T.w = width;
    T.shapes = shapes;
    T.stop_pow = stop_pow;
    T.tag = tag_frac;

    Work w{};
    w.cap = 1;
    w.nes = 1;
    w.Npad = ((n_grid + 127) / 128) * 128;
    w.Mpad = m_hi;
    w.pstride = T.P;
    w.n_items = 1;
    w.max_tiles = T.n_tiles;
    w.precision = BX_FP32;
    w.band = 8.0;
    w.watchdog_ns = 2000000000ull;
    w.toys = &scr->toy;
    w.toy_of = &scr->toy_of;
    w.theta = theta;
    w.tstride = T.P;
    w.col64 = scr->col64;
    w.colq = scr->colq;
    w.colf = scr->colf;
    w.colg = scr->colg;
    w.colS = scr->colS;
    w.colS32 = scr->colS32;
    w.colAl = scr->colAl;
    w.aW = scr->aW;
    w.colr = scr->colr;
    w.tile_cols = scr->tile_cols;
    w.cb_rows = scr->cb_rows;
    w.lam = lambda;   // written directly: [2][m_hi] with tag fractions, [m_hi] without
    w.status = &scr->status;
    w.err = &scr->err;
    w.units = &scr->units;
    w.count_units = 0;

    k_noalloc_begin<<<1, 1, 0, s>>>(T, scr);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_prep(w, 1, s);
    if (e == cudaSuccess) e = launch_fwd_f32(w, 1, T.n_tiles, T.has_tag, 0, s);
    if (e == cudaSuccess) {
        const int n = m_hi * (1 + T.has_tag);
        k_noalloc_end<<<(n + 255) / 256, 256, 0, s>>>(scr, lambda, n);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return bx_set_error(BX_ECUDA, "bx_spectra_noalloc: %s", cudaGetErrorString(e));
    return BX_OK;
}
