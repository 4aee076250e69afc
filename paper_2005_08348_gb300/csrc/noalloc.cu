// Force evaluation that allocates nothing (mdas_forces_noalloc).
//
// Some callers cannot allocate device memory while they run: code that works
// inside a fixed memory budget handed to it by a host application, code
// running between the allocations of another framework that owns the device
// heap, or a real-time loop that must not hit cudaMalloc's implicit device
// synchronisation.  This entry point evaluates the forces of one state from
// device buffers the caller already owns, using as scratch a fixed array that
// exists for as long as the library is loaded.
//
// Limits: at most NA_MAX_BEADS beads, NA_MAX_CELLS cells and NA_CAPC beads
// per cell.  Every call uses the same scratch array, so calls that overlap on
// the GPU (different streams, or different host threads) race and must be
// serialised by the caller.  The first call on a device looks up the array's
// device address (cudaGetSymbolAddress); make that first call before any
// stream capture.  Every call reads the device error word back and waits for
// its stream before it returns.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/mdas.h"
#include "host_params.h"
#include "mdas_dev.cuh"

using namespace mdas;

namespace {

constexpr int NA_MAX_BEADS = 16384;
constexpr int NA_MAX_CELLS = 2048;
constexpr int NA_CAPC = 64;
constexpr int NA_MAX_DEVICES = 64;

// scratch layout (byte offsets, each a multiple of 256)
constexpr size_t al(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t OFF_PARAMS = 0;
constexpr size_t OFF_COUNTERS = OFF_PARAMS + al(sizeof(Params));
constexpr size_t OFF_SYS = OFF_COUNTERS + al(sizeof(Counters));
constexpr size_t OFF_POS = OFF_SYS + al(sizeof(SysDev));
constexpr size_t OFF_FX = OFF_POS + al(16ull * NA_MAX_BEADS);
constexpr size_t OFF_FY = OFF_FX + al(8ull * NA_MAX_BEADS);
constexpr size_t OFF_FZ = OFF_FY + al(8ull * NA_MAX_BEADS);
constexpr size_t OFF_SIDX = OFF_FZ + al(8ull * NA_MAX_BEADS);
constexpr size_t OFF_COUNT = OFF_SIDX + al(4ull * NA_MAX_BEADS);
constexpr size_t OFF_CELLN = OFF_COUNT + al(4ull * NA_MAX_CELLS);
constexpr size_t OFF_TMP = OFF_CELLN + al(4ull * NA_MAX_CELLS);
constexpr size_t OFF_SORTED = OFF_TMP + al(4ull * NA_MAX_CELLS * NA_CAPC);
constexpr size_t OFF_SPOS = OFF_SORTED + al(4ull * NA_MAX_CELLS * NA_CAPC);
constexpr size_t OFF_BFORCE = OFF_SPOS + al(16ull * NA_MAX_CELLS * NA_CAPC);
constexpr size_t OFF_MAP_BEADS = OFF_BFORCE + al(32ull * NA_MAX_CELLS * NA_CAPC);
constexpr size_t OFF_MAP_CELLS = OFF_MAP_BEADS + al(8ull * (NA_MAX_BEADS / BEAD_BLOCK + 1));
constexpr size_t OFF_MAP_SORT = OFF_MAP_CELLS + al(8ull * NA_MAX_CELLS);
constexpr size_t OFF_MAP_SYS = OFF_MAP_SORT + al(8ull * (NA_MAX_CELLS / CELLS_PER_SORT_BLOCK + 1));
constexpr size_t NA_BYTES = OFF_MAP_SYS + al(8);

// the scratch: every GPU that loads the library holds it until exit (~8 MB)
static __device__ __align__(256) unsigned char g_na_scratch[NA_BYTES];

unsigned char *g_na_addr[NA_MAX_DEVICES];
std::mutex g_na_mu;

// failures are reported by status code only (no host heap use on this path)
inline mdas_status na_fail(mdas_status st, const char *) { return st; }

// fixed-point positions + lipid types (caller's device buffers) -> positions
// with the meta word; the block maps of one system (no thermostat block)
__global__ void k_na_prepare(const uint32_t *__restrict__ pos_fixed, const int32_t *__restrict__ ltype,
                             const Params *__restrict__ P, uint4 *__restrict__ pos, int water_bt, int *err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P->n) return;
    uint32_t m;
    if (i < P->n_lipid_beads) {
        const int l = i / P->bpl, k = i % P->bpl;
        int lt = ltype[l];
        if (lt < 0 || lt >= P->n_lt) {            // a type outside the table: flag it, read type 0
            atomicOr(err, ERR_BAD_INPUT);
            lt = 0;
        }
        const int bt = P->lbt[lt * 16 + k];
        m = meta_make(bt, bt, k, l + 1);
    } else {
        m = meta_make(water_bt, water_bt, 15, 0);
    }
    pos[i] = make_uint4(pos_fixed[3 * i], pos_fixed[3 * i + 1], pos_fixed[3 * i + 2], m);
}

__global__ void k_na_maps(int n, int n_cells, int2 *beads, int2 *cells, int2 *sortcells, int2 *syss) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k * BEAD_BLOCK < n) beads[k] = make_int2(0, k * BEAD_BLOCK);
    if (k < n_cells) cells[k] = make_int2(0, k);
    if (k * CELLS_PER_SORT_BLOCK < n_cells) sortcells[k] = make_int2(0, k * CELLS_PER_SORT_BLOCK);
    if (k == 0) syss[0] = make_int2(0, 0);
}

// the force-field parameters of a description: the tables mdas_create_system
// builds (one shared host function), within this entry point's limits
mdas_status na_params(const mdas_system_desc *d, Params &P) {
    if (d->n_beads <= 0 || d->n_beads > NA_MAX_BEADS) return na_fail(MDAS_ERR_INVALID_ARG, "forces_noalloc: too many beads");
    if (const char *why = fill_force_field(d, 0.0, P)) return na_fail(MDAS_ERR_INVALID_ARG, why);
    if (P.n_cells > NA_MAX_CELLS) return na_fail(MDAS_ERR_INVALID_ARG, "forces_noalloc: too many cells");
    P.capc = NA_CAPC;
    return MDAS_OK;
}

#define NACK(call)                                                                      \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) return na_fail(MDAS_ERR_CUDA, #call);                    \
    } while (0)

}  // namespace

extern "C" mdas_status mdas_forces_noalloc(const mdas_system_desc *d, const uint32_t *pos_fixed,
                                           const int32_t *lipid_type, double *f_out) {
    if (!d || !pos_fixed || !f_out || (d->n_lipids > 0 && !lipid_type))
        return na_fail(MDAS_ERR_INVALID_ARG, "forces_noalloc: NULL argument");
    Params P;
    mdas_status st = na_params(d, P);
    if (st != MDAS_OK) return st;
    cudaStream_t stream = (cudaStream_t)d->cuda_stream;

    // once per device (this device current): the device address of the scratch array
    int dev = 0;
    NACK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(MDAS_ERR_INVALID_ARG, "forces_noalloc: device index");
    unsigned char *base;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_addr[dev]) {
            void *ptr = nullptr;
            NACK(cudaGetSymbolAddress(&ptr, g_na_scratch));
            g_na_addr[dev] = (unsigned char *)ptr;
        }
        base = g_na_addr[dev];
    }
    NACK(setup_kernels());

    SysDev S;
    memset(&S, 0, sizeof(S));
    S.p = (const Params *)(base + OFF_PARAMS);
    S.c = (Counters *)(base + OFF_COUNTERS);
    S.pos = (uint4 *)(base + OFF_POS);
    S.fx = (long long *)(base + OFF_FX);
    S.fy = (long long *)(base + OFF_FY);
    S.fz = (long long *)(base + OFF_FZ);
    S.sidx = (int *)(base + OFF_SIDX);
    S.cell_count = (int *)(base + OFF_COUNT);
    S.cell_n = (int *)(base + OFF_CELLN);
    S.tmp_ids = (int *)(base + OFF_TMP);
    S.sorted_id = (int *)(base + OFF_SORTED);
    S.spos = (uint4 *)(base + OFF_SPOS);
    S.bforce = (void *)(base + OFF_BFORCE);
    S.n_bead_blocks = (P.n + BEAD_BLOCK - 1) / BEAD_BLOCK;

    // the previous call's contents stay in the array: clear what must start at zero
    NACK(cudaMemsetAsync(base + OFF_COUNTERS, 0, sizeof(Counters), stream));
    NACK(cudaMemsetAsync(base + OFF_COUNT, 0, 4ull * P.n_cells, stream));
    NACK(cudaMemcpyAsync(base + OFF_PARAMS, &P, sizeof(Params), cudaMemcpyHostToDevice, stream));
    NACK(cudaMemcpyAsync(base + OFF_SYS, &S, sizeof(SysDev), cudaMemcpyHostToDevice, stream));

    BlockMap beads, cells, sortcells, syss;
    beads.d = (int2 *)(base + OFF_MAP_BEADS);
    beads.n = S.n_bead_blocks;
    cells.d = (int2 *)(base + OFF_MAP_CELLS);
    cells.n = P.n_cells;
    sortcells.d = (int2 *)(base + OFF_MAP_SORT);
    sortcells.n = (P.n_cells + CELLS_PER_SORT_BLOCK - 1) / CELLS_PER_SORT_BLOCK;   // no thermostat block
    syss.d = (int2 *)(base + OFF_MAP_SYS);
    syss.n = 1;
    const int nmap = std::max(P.n_cells, S.n_bead_blocks);
    k_na_maps<<<(nmap + 127) / 128, 128, 0, stream>>>(P.n, P.n_cells, beads.d, cells.d, sortcells.d, syss.d);
    k_na_prepare<<<(P.n + 255) / 256, 256, 0, stream>>>(pos_fixed, lipid_type, S.p, S.pos, d->water_bead_type,
                                                         &S.c->err);

    LaunchCtx L;
    L.sys = (const SysDev *)(base + OFF_SYS);
    L.n_sys = 1;
    L.beads = &beads; L.cells = &cells; L.sortcells = &sortcells; L.syss = &syss;
    L.precision = d->precision;
    L.stream = stream;
    L.max_bead_blocks = S.n_bead_blocks;
    launch_cells(L);
    launch_pair(L, false, false, d->precision == MDAS_FP64);
    launch_total_force(L, f_out, 0);
    NACK(cudaGetLastError());
    int err = 0;
    NACK(cudaMemcpyAsync(&err, &S.c->err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    NACK(cudaStreamSynchronize(stream));
    if (err & ERR_BAD_INPUT) return na_fail(MDAS_ERR_INVALID_ARG, "forces_noalloc: lipid type out of range");
    // a cell over this entry point's fixed capacity is a size limit of the
    // call, not an instability of the state
    if (err & ERR_CELL_OVERFLOW)
        return na_fail(MDAS_ERR_INVALID_ARG, "forces_noalloc: more than 64 beads in a cell");
    if (err) return na_fail(MDAS_ERR_UNSTABLE, "forces_noalloc: device error flag");
    return MDAS_OK;
}
