// C ABI of the library (include/mdas.h): system lifetime, device memory,
// CUDA-graph replay of MD segments, batched exchange trials, MDAS moves and
// multi-system batches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/mdas.h"
#include "host_params.h"
#include "mdas_dev.cuh"

using namespace mdas;

namespace {

struct Batch {
    std::vector<mdas_system *> sys;
    SysDev *dsys = nullptr;
    BlockMap beads, cells, sortcells, syss, nlbeads, lsort;
    int precision = 0;
    cudaStream_t stream = nullptr;
    int max_bead_blocks = 1;
    int *dscratch = nullptr;      // [2]: pending sum, error or
    unsigned int *bticket = nullptr;   // last-block ticket of the step kernel over the batch
    void *rsync = nullptr;        // grid-barrier state of the persistent MD kernel (zeroed)
    void *part = nullptr;         // partition of the persistent kernel's groups among the systems
    size_t part_cap = 0;
    int part_groups = 0;          // groups the partition was made for (0: none made yet)
    bool persistent = true;       // MD in the persistent kernel (else separate kernel launches)
    int lanes = NL_LANES;         // list columns per bead of the batch's pair lists (all its systems agree)
    int trial_path = MDAS_TRIALS_AUTO;   // how batched exchange trials run (the first system's choice)
    size_t cap_sys = 0, cap_beads = 0, cap_cells = 0, cap_sort = 0;   // device capacity (refillable batches)
    size_t cap_nlb = 0, cap_ls = 0;
    LaunchCtx ctx() const;
};

std::string g_last_error;

// Pair-list geometry of a description: rl = rc + skin (limited so that every
// box edge holds 3 list-build cells), the list-build grid, and capacities from
// the densest list-build cell of the initial positions (a membrane patch may
// leave part of its box empty): a cell holds up to twice that count (at least
// four times the mean), a bead's list 1.5 times the number of beads within rl
// at that density, both multiples of 32.
struct ListDims {
    double rl;
    int ln[3], n_lcells, lcapc, lcap, npad;
};

// The fraction by which each box edge may shrink under pressure coupling
// (the cell grids are sized for it); 0 for a fixed box.
double grid_shrink(const mdas_system_desc *d) {
    if (!(d->tau_p > 0)) return 0.0;
    return d->box_margin > 0 ? std::min(d->box_margin, 0.5) : 0.05;
}

// Pair-list grid of a system whose box edges may shrink to (1 - shrink) of
// their length.
ListDims list_dims(const mdas_system_desc *d, double shrink = 0.0) {
    ListDims L;
    const double skin = d->list_skin > 0 ? d->list_skin : 0.35;
    const double f = 1.0 - shrink;
    const double lmin = std::min(d->box[0], std::min(d->box[1], d->box[2])) * f;
    L.rl = std::max(d->rc, std::min(d->rc + skin, lmin / 3.0));
    for (int k = 0; k < 3; ++k) L.ln[k] = std::max(3, (int)std::floor(d->box[k] * f / L.rl));
    L.n_lcells = L.ln[0] * L.ln[1] * L.ln[2];
    const int n = d->n_beads;
    std::vector<int> cnt(L.n_lcells, 0);
    int maxc = 0;
    for (int i = 0; i < n && d->pos; ++i) {
        int c[3];
        for (int k = 0; k < 3; ++k) {
            double f = d->pos[3 * i + k] / d->box[k];
            f -= std::floor(f);
            c[k] = std::min(L.ln[k] - 1, std::max(0, (int)(f * L.ln[k])));
        }
        maxc = std::max(maxc, ++cnt[(c[2] * L.ln[1] + c[1]) * L.ln[0] + c[0]]);
    }
    const double mean = (double)n / L.n_lcells;
    L.lcapc = std::max(32, (int)std::ceil(std::max(4.0 * mean, 2.0 * maxc) / 32.0) * 32);
    const double vol = d->box[0] * d->box[1] * d->box[2] * f * f * f;
    const double dens = std::max((double)n / vol, maxc / (vol / L.n_lcells));
    const double within = 4.0 / 3.0 * M_PI * L.rl * L.rl * L.rl * dens;
    L.lcap = std::max(64, (int)std::ceil(1.5 * within / 32.0) * 32);
    L.npad = (n + 31) / 32 * 32;
    return L;
}

}  // namespace

struct mdas_system {
    Params hp;
    SysDev hs;
    int n = 0, n_lip = 0, bpl = 0, precision = 0, water_bt = 0;
    cudaStream_t stream = nullptr;
    void *(*dev_alloc)(size_t, void *, void *) = nullptr;
    void (*dev_free)(void *, void *, void *) = nullptr;
    void *alloc_ctx = nullptr;
    void *arena = nullptr;
    size_t arena_bytes = 0;
    double *fout = nullptr;
    uint4 *rdf_info = nullptr;           // head-bead distribution: per lipid head and leaflet
    unsigned long long *rdf_hist = nullptr;
    int *rdf_nh = nullptr;
    std::unique_ptr<Batch> solo;
    std::string err;
    bool unstable = false;
    bool cells_valid = false;   // the cell list matches the current positions and types
    bool timing = false;
    bool partition = true;      // batches may give this system its own share of the persistent kernel's groups
    long long wave_beads = 0;   // a batch's MD runs in waves of systems of at most this many beads (0: all at once)
    int lanes = NL_LANES;       // list columns per bead this system's MD uses (mdas_set_list_lanes)
    int list_lanes = 0;         // the list columns its current pair list was built with (0: none yet)
    int trial_path = MDAS_TRIALS_AUTO;   // mdas_set_trial_path
    double pair_ms = 0.0;
    long long pair_launches = 0;
    long long kernel_launches = 0;   // kernel launches (graph kernel nodes included) that advanced this system
};

namespace {
LaunchCtx Batch::ctx() const {
    LaunchCtx L;
    L.sys = dsys; L.n_sys = (int)sys.size();
    L.beads = &beads; L.cells = &cells; L.sortcells = &sortcells; L.syss = &syss;
    L.nlbeads = &nlbeads; L.lsort = &lsort;
    L.precision = precision; L.stream = stream; L.max_bead_blocks = max_bead_blocks;
    L.lanes = lanes;
    L.bticket = bticket;
    L.soft = false;
    L.pc = false;
    for (auto *x : sys) {
        L.soft = L.soft || x->hp.sc_delta > 0.0;
        L.pc = L.pc || x->hp.pc_nst > 0;
    }
    return L;
}
}  // namespace

namespace {


std::map<std::vector<mdas_system *>, std::unique_ptr<Batch>> g_batches;

// The stream of systems created with cuda_stream == NULL: one non-blocking
// stream per process (graph capture is not possible on the legacy stream).
cudaError_t shared_stream(cudaStream_t *out) {
    static cudaStream_t st = nullptr;
    static cudaError_t err = cudaErrorNotReady;
    if (err == cudaErrorNotReady) err = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    *out = st;
    return err;
}

mdas_status fail(mdas_system *s, mdas_status st, const std::string &msg) {
    if (s) s->err = msg;
    g_last_error = msg;
    return st;
}

mdas_status cuda_fail(mdas_system *s, cudaError_t e, const char *where) {
    return fail(s, MDAS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(s, e_, #call);    \
    } while (0)

void *dalloc(mdas_system *s, size_t bytes) {
    void *p = nullptr;
    if (s->dev_alloc) p = s->dev_alloc(bytes, (void *)s->stream, s->alloc_ctx);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    return p;
}

void dfree(mdas_system *s, void *p) {
    if (!p) return;
    if (s->dev_free) s->dev_free(p, (void *)s->stream, s->alloc_ctx);
    else cudaFree(p);
}

void free_map(BlockMap &m) {
    if (m.d) cudaFree(m.d);
    m.d = nullptr;
    m.n = 0;
}

cudaError_t upload_map(BlockMap &m, const std::vector<int2> &v) {
    m.n = (int)v.size();
    cudaError_t e = cudaMalloc(&m.d, sizeof(int2) * std::max<size_t>(1, v.size()));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(m.d, v.data(), sizeof(int2) * v.size(), cudaMemcpyHostToDevice);
}

void destroy_batch(Batch *b) {
    free_map(b->beads); free_map(b->cells); free_map(b->sortcells); free_map(b->syss);
    free_map(b->nlbeads); free_map(b->lsort);
    if (b->dsys) cudaFree(b->dsys);
    if (b->dscratch) cudaFree(b->dscratch);
    if (b->bticket) cudaFree(b->bticket);
    if (b->rsync) cudaFree(b->rsync);
    if (b->part) cudaFree(b->part);
}

// block maps of a batch: per system its bead blocks, cells, cell groups of the
// cell-list finish (plus the thermostat block), step-kernel blocks and
// list-build place items (four cells each)
struct Maps {
    std::vector<int2> beads, cells, sortcells, syss, nlbeads, lsort;
    int lanes = NL_LANES;      // the batch's list columns per bead (step items of NL_BLOCK / lanes beads)
    void add(int k, const mdas_system *x);
};

void Maps::add(int k, const mdas_system *x) {
    for (int i = 0; i < x->n; i += BEAD_BLOCK) beads.push_back(make_int2(k, i));
    for (int c = 0; c < x->hp.n_cells; ++c) cells.push_back(make_int2(k, c));
    for (int c = 0; c < x->hp.n_cells; c += CELLS_PER_SORT_BLOCK) sortcells.push_back(make_int2(k, c));
    sortcells.push_back(make_int2(k, -1));   // the system's thermostat block
    syss.push_back(make_int2(k, 0));
    for (int i = 0; i < x->n; i += NL_BLOCK / lanes) nlbeads.push_back(make_int2(k, i));
    for (int c = 0; c < x->hp.n_lcells; c += CELLS_PER_SORT_BLOCK) lsort.push_back(make_int2(k, c));
}

mdas_status make_batch(const std::vector<mdas_system *> &v, std::unique_ptr<Batch> &out) {
    mdas_system *s = v[0];
    auto b = std::make_unique<Batch>();
    b->sys = v;
    b->precision = v[0]->precision;
    b->stream = v[0]->stream;
    b->lanes = v[0]->lanes;
    b->trial_path = v[0]->trial_path;
    std::vector<SysDev> hs;
    Maps mp;
    mp.lanes = b->lanes;
    for (int k = 0; k < (int)v.size(); ++k) {
        const mdas_system *x = v[k];
        if (x->precision != b->precision) return fail(s, MDAS_ERR_INVALID_ARG, "batch: systems differ in precision");
        if (x->stream != b->stream) return fail(s, MDAS_ERR_INVALID_ARG, "batch: systems differ in CUDA stream");
        if (x->lanes != b->lanes) return fail(s, MDAS_ERR_INVALID_ARG, "batch: systems differ in list lanes");
        hs.push_back(x->hs);
        mp.add(k, x);
        b->max_bead_blocks = std::max(b->max_bead_blocks, (x->n + BEAD_BLOCK - 1) / BEAD_BLOCK);
    }
    CK(cudaMalloc(&b->dsys, sizeof(SysDev) * hs.size()));
    CK(cudaMemcpy(b->dsys, hs.data(), sizeof(SysDev) * hs.size(), cudaMemcpyHostToDevice));
    CK(upload_map(b->beads, mp.beads));
    CK(upload_map(b->cells, mp.cells));
    CK(upload_map(b->sortcells, mp.sortcells));
    CK(upload_map(b->syss, mp.syss));
    CK(upload_map(b->nlbeads, mp.nlbeads));
    CK(upload_map(b->lsort, mp.lsort));
    CK(cudaMalloc(&b->dscratch, sizeof(int) * 4));
    CK(cudaMalloc(&b->bticket, sizeof(unsigned int)));
    CK(cudaMemset(b->bticket, 0, sizeof(unsigned int)));
    CK(cudaMalloc(&b->rsync, md_run_sync_bytes()));
    CK(cudaMemset(b->rsync, 0, md_run_sync_bytes()));
    out = std::move(b);
    return MDAS_OK;
}

// Refill a reusable batch with a new set of systems: device arrays only grow.
mdas_status refill_batch(Batch &b, const std::vector<mdas_system *> &v) {
    mdas_system *s = v[0];
    for (const mdas_system *x : v)             // checked before the batch changes
        if (x->precision != s->precision || x->stream != s->stream || x->lanes != s->lanes)
            return fail(s, MDAS_ERR_INVALID_ARG, "batch: systems differ in precision, stream or list lanes");
    b.sys = v;
    b.precision = v[0]->precision;
    b.stream = v[0]->stream;
    b.lanes = v[0]->lanes;
    b.trial_path = v[0]->trial_path;
    b.max_bead_blocks = 1;
    std::vector<SysDev> hs;
    Maps mp;
    mp.lanes = b.lanes;
    for (int k = 0; k < (int)v.size(); ++k) {
        const mdas_system *x = v[k];
        if (x->precision != b.precision || x->stream != b.stream || x->lanes != b.lanes)
            return fail(s, MDAS_ERR_INVALID_ARG, "batch: systems differ in precision, stream or list lanes");
        hs.push_back(x->hs);
        mp.add(k, x);
        b.max_bead_blocks = std::max(b.max_bead_blocks, (x->n + BEAD_BLOCK - 1) / BEAD_BLOCK);
    }
    std::vector<int2> &beads = mp.beads, &cells = mp.cells, &sortcells = mp.sortcells, &syss = mp.syss;
    auto grow = [&](void **ptr, size_t &cap, size_t need, size_t elem) -> cudaError_t {
        if (need <= cap && *ptr) return cudaSuccess;
        if (*ptr) cudaFree(*ptr);
        cap = std::max<size_t>(need * 2, 64);
        return cudaMalloc(ptr, cap * elem);
    };
    CK(grow((void **)&b.dsys, b.cap_sys, hs.size(), sizeof(SysDev)));
    CK(grow((void **)&b.beads.d, b.cap_beads, beads.size(), sizeof(int2)));
    CK(grow((void **)&b.cells.d, b.cap_cells, cells.size(), sizeof(int2)));
    CK(grow((void **)&b.sortcells.d, b.cap_sort, sortcells.size(), sizeof(int2)));
    CK(grow((void **)&b.nlbeads.d, b.cap_nlb, mp.nlbeads.size(), sizeof(int2)));
    CK(grow((void **)&b.lsort.d, b.cap_ls, mp.lsort.size(), sizeof(int2)));
    size_t cap_syss = 0;
    if (!b.syss.d) CK(grow((void **)&b.syss.d, cap_syss, 4096, sizeof(int2)));
    if (syss.size() > 4096) return fail(s, MDAS_ERR_INVALID_ARG, "batch: more than 4096 systems");
    if (!b.dscratch) CK(cudaMalloc(&b.dscratch, sizeof(int) * 4));
    if (!b.bticket) {
        CK(cudaMalloc(&b.bticket, sizeof(unsigned int)));
        CK(cudaMemset(b.bticket, 0, sizeof(unsigned int)));
    }
    if (!b.rsync) {
        CK(cudaMalloc(&b.rsync, md_run_sync_bytes()));
        CK(cudaMemset(b.rsync, 0, md_run_sync_bytes()));
    }
    CK(cudaMemcpyAsync(b.dsys, hs.data(), sizeof(SysDev) * hs.size(), cudaMemcpyHostToDevice, b.stream));
    CK(cudaMemcpyAsync(b.beads.d, beads.data(), sizeof(int2) * beads.size(), cudaMemcpyHostToDevice, b.stream));
    CK(cudaMemcpyAsync(b.cells.d, cells.data(), sizeof(int2) * cells.size(), cudaMemcpyHostToDevice, b.stream));
    CK(cudaMemcpyAsync(b.sortcells.d, sortcells.data(), sizeof(int2) * sortcells.size(), cudaMemcpyHostToDevice, b.stream));
    CK(cudaMemcpyAsync(b.syss.d, syss.data(), sizeof(int2) * syss.size(), cudaMemcpyHostToDevice, b.stream));
    CK(cudaMemcpyAsync(b.nlbeads.d, mp.nlbeads.data(), sizeof(int2) * mp.nlbeads.size(), cudaMemcpyHostToDevice, b.stream));
    CK(cudaMemcpyAsync(b.lsort.d, mp.lsort.data(), sizeof(int2) * mp.lsort.size(), cudaMemcpyHostToDevice, b.stream));
    CK(cudaStreamSynchronize(b.stream));   // the host vectors go out of scope
    b.beads.n = (int)beads.size();
    b.cells.n = (int)cells.size();
    b.sortcells.n = (int)sortcells.size();
    b.syss.n = (int)syss.size();
    b.nlbeads.n = (int)mp.nlbeads.size();
    b.lsort.n = (int)mp.lsort.size();
    b.part_groups = 0;                     // the partition is made again for the new systems
    return MDAS_OK;
}

// ------------------------------------------------------------ step bodies
mdas_status build_cells(mdas_system *s, Batch &b) {
    launch_cells(b.ctx());
    for (auto *x : b.sys) x->cells_valid = true;
    return MDAS_OK;
}

__global__ void k_batch_status(const SysDev *__restrict__ sys, int n, int *out) {
    int pend = 0, err = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) { pend += sys[k].c->pending; err |= sys[k].c->err; }
    for (int o = 16; o > 0; o >>= 1) {
        pend += __shfl_xor_sync(0xffffffffu, pend, o);
        err |= __shfl_xor_sync(0xffffffffu, err, o);
    }
    if (threadIdx.x == 0) { out[0] = pend; out[1] = err; }
}

mdas_status batch_status(mdas_system *s, Batch &b, int *pending, int *err) {
    k_batch_status<<<1, 32, 0, b.stream>>>(b.dsys, (int)b.sys.size(), b.dscratch);
    int h[2];
    CK(cudaMemcpyAsync(h, b.dscratch, sizeof(h), cudaMemcpyDeviceToHost, b.stream));
    CK(cudaStreamSynchronize(b.stream));
    *pending = h[0];
    *err = h[1];
    return MDAS_OK;
}

mdas_status check_err(mdas_system *s, Batch &b) {
    int pend, err;
    mdas_status st = batch_status(s, b, &pend, &err);
    if (st != MDAS_OK) return st;
    if (err) {
        for (auto *x : b.sys) x->unstable = true;
        std::string why;
        if (err & ERR_NONFINITE) why += " non-finite velocity;";
        if (err & ERR_CELL_OVERFLOW) why += " a cell holds more beads than its capacity;";
        if (err & ERR_TIMEOUT) why += " bounded wait expired;";
        if (err & ERR_ROUNDS) why += " exchange rounds exhausted;";
        if (err & ERR_BOX) why += " the box shrank below what the cell grids allow;";
        if (err & ERR_BOUNDS) why += " an index outside its array (checked build);";
        // a wait that gave up left the state partly advanced: refused like an
        // unstable one, reported as the timeout it was
        return fail(s, (err & ERR_TIMEOUT) ? MDAS_ERR_TIMEOUT : MDAS_ERR_UNSTABLE, "unstable:" + why);
    }
    return MDAS_OK;
}

// Timing of the MD kernels: events around each launch, read after the segment.
struct SegTimer {
    bool on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> evs;
    std::vector<long long> steps;
    cudaError_t begin(cudaStream_t st, long long n) {
        if (!on) return cudaSuccess;
        cudaEvent_t e0, e1;
        cudaError_t e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e != cudaSuccess) return e;
        evs.push_back({e0, e1});
        steps.push_back(n);
        return cudaEventRecord(e0, st);
    }
    cudaError_t end(cudaStream_t st) { return on ? cudaEventRecord(evs.back().second, st) : cudaSuccess; }
    cudaError_t collect(Batch &b) {
        if (evs.empty()) return cudaSuccess;
        cudaError_t e = cudaStreamSynchronize(b.stream);
        for (size_t k = 0; k < evs.size() && e == cudaSuccess; ++k) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, evs[k].first, evs[k].second);
            for (auto *x : b.sys) { x->pair_ms += ms; x->pair_launches += steps[k]; }
        }
        for (auto &ev : evs) { cudaEventDestroy(ev.first); cudaEventDestroy(ev.second); }
        evs.clear();
        return e;
    }
};

__global__ void k_run_abort(void *sync, int nbytes, const SysDev *__restrict__ sys, int n_sys, SysBar *bars) {
    // a persistent launch that gave up at a barrier: every system of the
    // batch records it, and the barrier state is cleared for the next launch
    const int *w = (const int *)sync;
    const int ab = w[2];
    if (ab == 0) return;
    for (int q = threadIdx.x; q < n_sys; q += blockDim.x) {
        atomicOr(&sys[q].c->err, ab);
        if (bars) bars[q].count = bars[q].base = 0u;
    }
    __syncthreads();
    if (threadIdx.x == 0) memset(sync, 0, nbytes);
}

// The partition of a persistent launch's groups among the systems of a
// batch (partitioned mode): groups in proportion to each system's step
// items, at least one each; false when the batch does not need it (one
// system, or every step item has a group of its own) or cannot have it
// (more systems than groups).
mdas_status make_partition(mdas_system *s, Batch &b, int groups, bool *use) {
    const int n = (int)b.sys.size();
    *use = false;
    std::vector<int> items(n);
    long long total = 0;
    for (int q = 0; q < n; ++q) {
        items[q] = (b.sys[q]->n + NL_BLOCK / b.lanes - 1) / (NL_BLOCK / b.lanes);
        total += items[q];
    }
    if (n < 2 || n > groups / 2 || total + (long long)(TRIAL_PARTS + 1) * n <= groups) return MDAS_OK;
    for (auto *x : b.sys)
        if (!x->partition) return MDAS_OK;
    *use = true;
    if (b.part_groups == groups) return MDAS_OK;
    std::vector<int> ng(n);
    int used = 0;
    for (int q = 0; q < n; ++q) {
        ng[q] = std::max(1, (int)((long long)groups * items[q] / total));
        used += ng[q];
    }
    while (used > groups) {                // take back from the system with the fewest items per group
        int best = -1;
        for (int q = 0; q < n; ++q)
            if (ng[q] > 1 && (best < 0 || (double)items[q] / ng[q] < (double)items[best] / ng[best])) best = q;
        if (best < 0) { *use = false; return MDAS_OK; }
        --ng[best]; --used;
    }
    while (used < groups) {                // give to the system with the most items per group
        int best = 0;
        for (int q = 1; q < n; ++q)
            if ((double)items[q] / ng[q] > (double)items[best] / ng[best]) best = q;
        ++ng[best]; ++used;
    }
    const PartLayout pl = part_layout(n, groups);
    std::vector<char> host(pl.bytes, 0);
    SysRange *r = (SysRange *)(host.data() + pl.ranges);
    int *gs = (int *)(host.data() + pl.gsys);
    int g0 = 0, nl0 = 0, bd0 = 0, ls0 = 0;
    for (int q = 0; q < n; ++q) {
        const mdas_system *x = b.sys[q];
        r[q].g0 = g0; r[q].ng = ng[q];
        r[q].nl0 = nl0; r[q].nln = (x->n + NL_BLOCK / b.lanes - 1) / (NL_BLOCK / b.lanes);
        r[q].bd0 = bd0; r[q].bdn = (x->n + BEAD_BLOCK - 1) / BEAD_BLOCK;
        r[q].ls0 = ls0; r[q].lsn = (x->hp.n_lcells + CELLS_PER_SORT_BLOCK - 1) / CELLS_PER_SORT_BLOCK;
        for (int k = 0; k < ng[q]; ++k) gs[g0 + k] = q;
        g0 += ng[q]; nl0 += r[q].nln; bd0 += r[q].bdn; ls0 += r[q].lsn;
    }
    if (nl0 != b.nlbeads.n || bd0 != b.beads.n || ls0 != b.lsort.n)
        return fail(s, MDAS_ERR_INVALID_ARG, "batch: block maps do not match the partition");
    if (pl.bytes > b.part_cap) {
        if (b.part) cudaFree(b.part);
        b.part = nullptr;
        CK(cudaMalloc(&b.part, pl.bytes));
        b.part_cap = pl.bytes;
    }
    CK(cudaMemcpyAsync(b.part, host.data(), pl.bytes, cudaMemcpyHostToDevice, b.stream));
    CK(cudaStreamSynchronize(b.stream));
    b.part_groups = groups;
    return MDAS_OK;
}

// A pair list laid out for another step shape is built again for this
// batch's: its systems' lists are marked stale (the next build, in the MD
// launch or launch_nl_build, makes them).
mdas_status lists_for_shape(mdas_system *s, Batch &b) {
    static const int one = 1;
    for (auto *x : b.sys)
        if (x->list_lanes != b.lanes) {
            CK(cudaMemcpyAsync(&x->hs.c->nl_stale, &one, sizeof(int), cudaMemcpyHostToDevice, b.stream));
            x->list_lanes = b.lanes;
        }
    return MDAS_OK;
}

// n_steps MD steps on a batch; after every swap_every-th step one trial.
// Segments of up to MAX_DRAW_STEPS - 1 steps: the thermostat variates of the
// segment, the first step's factor, then the persistent kernel (or, when it
// cannot run or plain launches are asked for, the separate kernels step by
// step, with the same arithmetic).
mdas_status run_md(mdas_system *s, Batch &b, long long n_steps, int swap_every, bool lambda = false,
                   bool check = true, int lam_M = 0, double dlam = 0.0, long long lam_base = 0) {
    if (n_steps <= 0) return MDAS_OK;
    const bool trial = swap_every > 0;
    SegTimer tm;
    for (auto *x : b.sys) tm.on = tm.on || x->timing;
    for (auto *x : b.sys) x->cells_valid = false;
    {
        mdas_status st = lists_for_shape(s, b);
        if (st != MDAS_OK) return st;
    }
    LaunchCtx L = b.ctx();
    const int run_mode = !lambda ? (L.pc ? 3 : 0) : L.soft ? 2 : 1;
    const bool persistent = b.persistent && md_run_blocks(b.precision, run_mode, b.lanes) > 0;
    if (persistent) {
        bool use = false;
        mdas_status st = make_partition(s, b, md_run_groups(b.precision, run_mode, b.lanes), &use);
        if (st != MDAS_OK) return st;
        if (use) {
            L.part = b.part;
            L.part_groups = b.part_groups;
        }
    }
    // segments of at most MAX_DRAW_STEPS - 1 steps (the precomputed thermostat
    // variates); a segment starting at step k0 has its trials after local
    // steps s with (k0 + s + 1) % swap_every == 0
    const long long seg = MAX_DRAW_STEPS - 1;
    long long launches = 0;
    // pressure coupling: segments also end where a box update is due (a step
    // counter that is a multiple of nstpcouple), which follows the segment;
    // the coupled systems of a batch must share nstpcouple and the phase
    long long pc_nst = 0, pc_phase = 0;
    if (L.pc && !lambda) {
        for (auto *x : b.sys) {
            if (x->hp.pc_nst <= 0) continue;
            unsigned long long st = 0;
            CK(cudaMemcpyAsync(&st, &x->hs.c->step, sizeof(st), cudaMemcpyDeviceToHost, b.stream));
            CK(cudaStreamSynchronize(b.stream));
            const long long ph = (long long)(st % (unsigned long long)x->hp.pc_nst);
            if (pc_nst == 0) {
                pc_nst = x->hp.pc_nst;
                pc_phase = ph;
            } else if (pc_nst != x->hp.pc_nst || ph != pc_phase) {
                return fail(s, MDAS_ERR_INVALID_ARG, "md: pressure-coupled systems of a batch at different coupling phases");
            }
        }
    }
    for (long long k0 = 0, n = 0; k0 < n_steps; k0 += n) {
        n = std::min(seg, n_steps - k0);
        if (pc_nst > 0) n = std::min(n, pc_nst - (pc_phase + k0) % pc_nst);
        launch_thermo_draws(L, (int)std::min<long long>(n + 1, MAX_DRAW_STEPS));
        launch_thermostat(L);
        launches += 2;
        if (persistent) {
            CK(tm.begin(b.stream, n));
            CK(launch_md_run(L, lambda, (int)n, swap_every, trial ? (int)(k0 % swap_every) : 0, lam_M,
                             (int)(lam_base + k0), dlam, b.rsync));
            CK(tm.end(b.stream));
            k_run_abort<<<1, 32, 0, b.stream>>>(b.rsync, (int)md_run_sync_bytes(), b.dsys, (int)b.sys.size(),
                                                 L.part ? (SysBar *)((char *)L.part + part_layout((int)b.sys.size(),
                                                          L.part_groups).bars) : nullptr);
            launches += 1;
            if (pc_nst > 0) { launch_pcouple(L); ++launches; }
            continue;
        }
        // the same order as the persistent kernel: a build for lists made
        // stale outside, then per step: step, build after a violation, trial
        launch_nl_build(L);
        launches += 4;
        for (long long k = 0; k < n; ++k) {
            CK(tm.begin(b.stream, 1));
            launch_nl_step(L, lambda);
            CK(tm.end(b.stream));
            launch_nl_build(L);
            launches += 5;
            if (trial && (k0 + k + 1) % swap_every == 0) { launch_trial_nl(L); ++launches; }
            if (lam_M > 0 && (lam_base + k0 + k + 1) % lam_M == 0) {
                // the end of a lambda block: its work term, then the next lambda
                const long long blk = (lam_base + k0 + k + 1) / lam_M;       // lambda blocks done
                launch_mdas_dE_nl(L, (double)(blk - 1) * dlam, (double)blk * dlam, dlam);
                launch_mdas_set_lambda(L, (double)blk * dlam, 1);
                launches += 3;
            }
        }
        if (pc_nst > 0) { launch_pcouple(L); ++launches; }
    }
    if (pc_nst > 0) {
        // the host copy of the box-derived parameters
        for (auto *x : b.sys)
            if (x->hp.pc_nst > 0) CK(cudaMemcpyAsync(&x->hp, x->hs.p, sizeof(Params), cudaMemcpyDeviceToHost, b.stream));
        CK(cudaStreamSynchronize(b.stream));
    }
    for (auto *x : b.sys) x->kernel_launches += launches;
    CK(cudaGetLastError());
    CK(tm.collect(b));
    return check ? check_err(s, b) : MDAS_OK;
}

// n exchange trials per system of a batch with sequential semantics.
// The way a batch runs its exchange trials: its first system's choice, or
// for MDAS_TRIALS_AUTO one after another from the pair lists (measured
// faster for small and large bilayers alike: 64 replicas of 128-2048 lipids,
// 100 trials each, 1.8 against 7.1 ms; a 4608-lipid bilayer, 1024 trials,
// 104k against 72k trials/s) unless a system has pressure coupling, whose
// lists may predate the last box update.
int trial_path_of(const Batch &b, int) {
    if (b.trial_path != MDAS_TRIALS_AUTO) return b.trial_path;
    for (const mdas_system *x : b.sys)
        if (x->hp.pc_nst > 0) return MDAS_TRIALS_SPECULATIVE;
    return MDAS_TRIALS_SEQUENTIAL;
}

// n exchange trials of every system of a batch, one after another from the
// pair lists (the trial the persistent kernel runs after an MD step): one
// launch per trial with every system's 16 parts, no speculation and no
// host round trip; the lists are built first where stale.
mdas_status run_trials_nl(mdas_system *s, Batch &b, int n) {
    mdas_status st = lists_for_shape(s, b);
    if (st != MDAS_OK) return st;
    LaunchCtx L = b.ctx();
    launch_nl_build(L);
    for (int t = 0; t < n; ++t) launch_trial_nl(L);
    for (auto *x : b.sys) x->cells_valid = false;   // the cell-ordered copy keeps the old types
    CK(cudaGetLastError());
    return check_err(s, b);
}

mdas_status run_trials(mdas_system *s, Batch &b, int n, int *rounds_out) {
    if (trial_path_of(b, n) == MDAS_TRIALS_SEQUENTIAL) {
        if (rounds_out) *rounds_out = n;
        return run_trials_nl(s, b, n);
    }
    LaunchCtx L = b.ctx();
    mdas_status st0 = build_cells(s, b);
    if (st0 != MDAS_OK) return st0;
    int rounds = 0;
    for (int done = 0; done < n;) {
        const int m = std::min(n - done, MAX_ROUND_TRIALS);
        launch_swap_propose(L, m);
        for (int r = 0;; ++r) {
            if (r > m + 1) return fail(s, MDAS_ERR_TIMEOUT, "exchange trials: round limit reached");
            launch_swap_dE(L, m);
            launch_swap_resolve(L, m);
            ++rounds;
            int pend = 0, err = 0;
            mdas_status st = batch_status(s, b, &pend, &err);
            if (st != MDAS_OK) return st;
            if (pend == 0) break;
        }
        done += m;
    }
    for (auto *x : b.sys) x->cells_valid = true;
    CK(cudaGetLastError());
    if (rounds_out) *rounds_out = rounds;
    return check_err(s, b);
}

}  // namespace

namespace mdas {

const char *fill_force_field(const mdas_system_desc *d, double shrink, Params &P) {
    const int n = d->n_beads, nl = d->n_lipids, bpl = d->beads_per_lipid, nbt = d->n_bead_types, nlt = d->n_lipid_types;
    if (n <= 0 || nl < 0 || bpl <= 0 || bpl > MAXT || nbt <= 0 || nbt > MAXT || nlt <= 0 || nlt > MAXT ||
        nl * bpl > n || nl >= (1 << 20) || n > (1 << 28))
        return "sizes out of range";
    if (!d->lipid_bead_type || !d->eps || !d->sigma || !d->charge) return "missing array";
    if (d->water_bead_type < 0 || d->water_bead_type >= nbt) return "water type";
    if (!(d->rc > 0) || !(d->eps_r > 0)) return "rc, eps_r";
    if (d->n_bonds < 0 || d->n_angles < 0 || (d->n_bonds && !d->bonds) || (d->n_angles && !d->angles)) return "topology";
    if (d->precision != MDAS_FP32 && d->precision != MDAS_FP64) return "precision";
    memset(&P, 0, sizeof(P));
    for (int k = 0; k < 3; ++k) {
        if (!(d->box[k] > 0)) return "box";
        P.nc[k] = (int)std::floor(d->box[k] * (1.0 - shrink) / d->rc);
        if (P.nc[k] < 3) return "every box edge must be >= 3 rc (with the margin)";
    }
    for (int k = 0; k < nlt * bpl; ++k)
        if (d->lipid_bead_type[k] < 0 || d->lipid_bead_type[k] >= nbt) return "lipid bead type";
    P.n = n; P.n_lip = nl; P.bpl = bpl; P.n_bt = nbt; P.n_lt = nlt; P.n_lipid_beads = nl * bpl;
    P.n_cells = P.nc[0] * P.nc[1] * P.nc[2];
    P.rc = d->rc; P.rc2 = d->rc * d->rc;
    P.dt = d->dt;
    for (int k = 0; k < 3; ++k) box_params(P, k, d->box[k]);
    P.krf = d->eps_rf <= 0 ? 1.0 / (2.0 * d->rc * d->rc * d->rc)
                           : (d->eps_rf - d->eps_r) / ((2.0 * d->eps_rf + d->eps_r) * d->rc * d->rc * d->rc);
    P.crf = 1.0 / d->rc + P.krf * d->rc * d->rc;
    for (int k = 0; k < 3; ++k) P.cwu[k] = (unsigned long long)(4294967296.0 / P.nc[k]);
    // float cull bounds: every pair with r^2 < rc^2 passes rc2f; pairs in
    // [rc2f_lo, rc2f) are re-decided exactly from integer offsets
    P.rc2f = std::nextafter((float)(P.rc2 * (1.0 + 1e-5)), 1e30f);
    P.rc2f_lo = (float)(P.rc2 * (1.0 - 1e-5));
    P.krf2f = (float)(2.0 * P.krf);
    P.kb = d->kb; P.b0 = d->b0; P.kth = d->ktheta; P.cos0 = std::cos(d->theta0_deg * M_PI / 180.0);
    P.precision = d->precision;
    const double rc6 = std::pow(d->rc, 6);
    for (int a = 0; a < nbt; ++a)
        for (int b = 0; b < nbt; ++b) {
            const double e = d->eps[a * nbt + b], sg = d->sigma[a * nbt + b];
            const double s6 = std::pow(sg, 6);
            const int x = a * 16 + b;
            P.c12[x] = 4.0 * e * s6 * s6;
            P.c6[x] = 4.0 * e * s6;
            P.ush[x] = P.c12[x] / (rc6 * rc6) - P.c6[x] / rc6;
            P.qq[x] = COUL * d->charge[a] * d->charge[b] / d->eps_r;
            P.f12f[x] = (float)(12.0 * P.c12[x]);
            P.f6f[x] = (float)(6.0 * P.c6[x]);
            P.qqf[x] = (float)P.qq[x];
        }
    for (int lt = 0; lt < nlt; ++lt)
        for (int k = 0; k < bpl; ++k) P.lbt[lt * 16 + k] = (uint8_t)d->lipid_bead_type[lt * bpl + k];
    for (int b = 0; b < d->n_bonds; ++b) {
        const int p = d->bonds[2 * b], q = d->bonds[2 * b + 1];
        if (p < 0 || q < 0 || p >= bpl || q >= bpl || p == q || P.nbond[p] >= 4 || P.nbond[q] >= 4)
            return "bond (at most 4 per bead)";
        P.excl[p] |= (uint16_t)(1u << q);
        P.excl[q] |= (uint16_t)(1u << p);
        P.bpart[p][P.nbond[p]++] = (int8_t)q;
        P.bpart[q][P.nbond[q]++] = (int8_t)p;
    }
    for (int a = 0; a < d->n_angles; ++a) {
        const int t3[3] = {d->angles[3 * a], d->angles[3 * a + 1], d->angles[3 * a + 2]};
        for (int r = 0; r < 3; ++r) {
            const int k = t3[r];
            if (k < 0 || k >= bpl || P.nang[k] >= 8) return "angle (at most 8 per bead)";
            for (int c = 0; c < 3; ++c) P.ang[k][P.nang[k]][c] = (int8_t)t3[c];
            P.nang[k]++;
        }
    }
    // bonded partners of each local index (the beads its bonded terms read)
    memset(P.pidx, -1, sizeof(P.pidx));
    for (int k = 0; k < bpl; ++k) {
        auto add = [&](int q) {
            if (q == k || P.pidx[k][q] >= 0) return true;
            if (P.npart[k] >= NL_PART) return false;
            P.pidx[k][q] = (int8_t)P.npart[k];
            P.part[k][P.npart[k]++] = (int8_t)q;
            return true;
        };
        bool ok = true;
        for (int b = 0; b < P.nbond[k]; ++b) ok = ok && add(P.bpart[k][b]);
        for (int a = 0; a < P.nang[k]; ++a)
            for (int c = 0; c < 3; ++c) ok = ok && add(P.ang[k][a][c]);
        if (!ok) return "a bead has more than 8 bonded partners";
    }
    return nullptr;
}

}  // namespace mdas

// =================================================================== ABI

extern "C" {

const char *mdas_status_string(mdas_status st) {
    switch (st) {
        case MDAS_OK: return "ok";
        case MDAS_ERR_INVALID_ARG: return "invalid argument";
        case MDAS_ERR_OOM: return "out of device memory";
        case MDAS_ERR_CUDA: return "CUDA error";
        case MDAS_ERR_UNSTABLE: return "unstable state";
        case MDAS_ERR_TIMEOUT: return "timeout";
        case MDAS_ERR_BUSY: return "busy";
    }
    return "unknown";
}

const char *mdas_last_error(const mdas_system *s) { return s ? s->err.c_str() : g_last_error.c_str(); }

mdas_status mdas_create_system(const mdas_system_desc *d, mdas_system **out) {
    mdas_system *s = nullptr;
    if (!d || !out) return fail(nullptr, MDAS_ERR_INVALID_ARG, "create: NULL argument");
    *out = nullptr;
    const int n = d->n_beads, nl = d->n_lipids, bpl = d->beads_per_lipid, nlt = d->n_lipid_types;
    // pressure coupling: the cell grids hold for every edge down to (1 - shrink) of its length
    const bool pcouple = d->tau_p > 0;
    const double shrink = grid_shrink(d);
    Params P;
    if (const char *why = fill_force_field(d, shrink, P)) return fail(nullptr, MDAS_ERR_INVALID_ARG, std::string("create: ") + why);
    if (!d->pos || !d->lipid_type) return fail(nullptr, MDAS_ERR_INVALID_ARG, "create: missing array");
    if (!(d->mass > 0) || !(d->dt > 0) || !(d->temperature >= 0))
        return fail(nullptr, MDAS_ERR_INVALID_ARG, "create: rc, eps_r, mass, dt, temperature");
    if (pcouple && !(d->compressibility >= 0 && std::isfinite(d->p_ref) && std::isfinite(d->tau_p)))
        return fail(nullptr, MDAS_ERR_INVALID_ARG, "create: pressure coupling parameters");
    if ((long long)P.nc[0] * P.nc[1] * P.nc[2] > (1 << 26)) return fail(nullptr, MDAS_ERR_INVALID_ARG, "create: too many cells");
    for (int l = 0; l < nl; ++l) {
        if (d->lipid_first_bead && d->lipid_first_bead[l] != l * bpl)
            return fail(nullptr, MDAS_ERR_INVALID_ARG, "create: lipid l must own beads [l*bpl, (l+1)*bpl)");
        if (d->lipid_type[l] < 0 || d->lipid_type[l] >= nlt) return fail(nullptr, MDAS_ERR_INVALID_ARG, "create: lipid type");
    }

    {
        cudaError_t e = setup_kernels();
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "create: kernel setup");
    }
    cudaStream_t stream = (cudaStream_t)d->cuda_stream;
    if (!stream) {
        cudaError_t e = shared_stream(&stream);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "create: stream");
    }
    s = new mdas_system();
    s->n = n; s->n_lip = nl; s->bpl = bpl; s->precision = d->precision; s->water_bt = d->water_bead_type;
    s->stream = stream;
    s->dev_alloc = d->dev_alloc; s->dev_free = d->dev_free; s->alloc_ctx = d->alloc_ctx;
    if ((s->dev_alloc == nullptr) != (s->dev_free == nullptr)) {
        delete s;
        return fail(nullptr, MDAS_ERR_INVALID_ARG, "create: dev_alloc and dev_free go together");
    }

    // ---- parameters: the force field, then capacities, pair list, thermostat
    s->hp = P;
    {   // cell capacity: four times the mean occupancy, at least 32, a multiple of 32
        const double mean = (double)n / P.n_cells;
        P.capc = std::max(32, (int)std::ceil(4.0 * mean / 32.0) * 32);
        if (P.capc > 1024) {
            delete s;
            return fail(nullptr, MDAS_ERR_INVALID_ARG, "create: more than 256 beads per cell on average");
        }
    }
    {   // pair list
        const ListDims ld = list_dims(d, shrink);
        P.rl = ld.rl;
        P.rl2 = P.rl * P.rl;
        P.rl2f = std::nextafter((float)(P.rl2 * (1.0 + 1e-5)), 1e30f);
        P.dmax2f = list_dmax2f(P.rl, d->rc, 1.0);      // a bead may move (rl - rc) / 2 before a rebuild
        for (int k = 0; k < 3; ++k) {
            P.ln[k] = ld.ln[k];
            P.lcwu[k] = (unsigned long long)(4294967296.0 / ld.ln[k]);
        }
        P.n_lcells = ld.n_lcells;
        for (int k = 0; k < 3; ++k) P.pc_lmin[k] = std::max(P.nc[k] * d->rc, ld.ln[k] * P.rl);
        P.lcapc = ld.lcapc;
        if (P.lcapc > NLB_BEADS * 32767) {     // a cell's build tasks are counted in 15 bits
            delete s;
            return fail(nullptr, MDAS_ERR_INVALID_ARG, "create: too many beads in a list-build cell");
        }
        P.lcap = ld.lcap;
        P.npad = ld.npad;
        P.mark_words = (n + NL_BEADS_MIN - 1) / NL_BEADS_MIN / 32 + 1;
        if (P.lcapc > 4096 || P.lcap > 4096) {
            delete s;
            return fail(nullptr, MDAS_ERR_INVALID_ARG, "create: density too high for the pair list");
        }
    }
    if (pcouple) {
        const double beta = d->compressibility > 0 ? d->compressibility : 3e-4;
        P.pc_nst = d->nstpcouple > 0 ? d->nstpcouple : 10;
        P.pc_pref = d->p_ref;
        P.pc_wc = 4.0 * M_PI * M_PI * beta / (3.0 * d->tau_p * d->tau_p);
    }
    P.therm_c = d->tau_t > 0 ? std::exp(-d->dt / d->tau_t) : 1.0;
    P.tau_t = d->tau_t; P.mass = d->mass; P.kT = BOLTZ * d->temperature;
    P.dt_over_m = d->dt / d->mass;
    P.dt_over_mf = (float)P.dt_over_m;
    P.massf = (float)d->mass;
    P.nf[0] = 3 * nl * bpl; P.nf[1] = 3 * (n - nl * bpl);
    for (int g = 0; g < 2; ++g) P.ktarget[g] = 0.5 * P.nf[g] * P.kT;
    P.key0 = (uint32_t)d->seed ^ d->system_id;
    P.key1 = (uint32_t)(d->seed >> 32);
    s->hp = P;

    // ---- device memory: one arena
    const int nbb = (n + BEAD_BLOCK - 1) / BEAD_BLOCK;
    const size_t nslot = (size_t)P.n_cells * P.capc;
    const size_t vsz = d->precision == MDAS_FP64 ? 32 : 16;
    struct Item { void **ptr; size_t bytes; };
    SysDev &H = s->hs;
    memset(&H, 0, sizeof(H));
    Params *dp = nullptr; Counters *dc = nullptr;
    std::vector<Item> items = {
        {(void **)&dp, sizeof(Params)}, {(void **)&dc, sizeof(Counters)},
        {(void **)&H.pos, 16ull * n}, {(void **)&H.vel, vsz * n},
        {(void **)&H.fx, 8ull * n}, {(void **)&H.fy, 8ull * n}, {(void **)&H.fz, 8ull * n},
        {(void **)&H.ltype, 4ull * std::max(nl, 1)},
        {(void **)&H.cell_count, 4ull * P.n_cells}, {(void **)&H.cell_n, 4ull * P.n_cells},
        {(void **)&H.tmp_ids, 4ull * nslot}, {(void **)&H.sorted_id, 4ull * nslot}, {(void **)&H.sidx, 4ull * n},
        {(void **)&H.spos, 16ull * nslot}, {(void **)&H.bforce, vsz * nslot},
        {(void **)&H.ke_part, 16ull * P.n_cells}, {(void **)&H.bpart, 24ull * nbb}, {(void **)&H.epart, 32ull * P.n_cells},
        {(void **)&H.pos_snap, 16ull * n}, {(void **)&H.vel_snap, vsz * n},
        {(void **)&H.ltype_snap, 4ull * std::max(nl, 1)},
        {(void **)&H.tprop, 16ull * MAX_ROUND_TRIALS}, {(void **)&H.tu, 8ull * MAX_ROUND_TRIALS},
        {(void **)&H.tdE, 8ull * 9 * MAX_ROUND_TRIALS}, {(void **)&H.tstate, 4ull * MAX_ROUND_TRIALS},
        {(void **)&H.conflict, 4ull * MAX_ROUND_TRIALS * (MAX_ROUND_TRIALS / 32)},
        {(void **)&H.lbox, 32ull * MAX_ROUND_TRIALS}, {(void **)&H.lhalf, 32ull * MAX_ROUND_TRIALS},
        {(void **)&H.log, sizeof(TrialRec) * (size_t)LOG_CAP}, {(void **)&H.result, 8ull * 64},
        {(void **)&H.tdraw, sizeof(double2) * 2ull * MAX_DRAW_STEPS},
        {(void **)&s->fout, 24ull * n},
        {(void **)&s->rdf_info, 16ull * std::max(nl, 1)}, {(void **)&s->rdf_hist, 16ull * RDF_MAX_BINS},
        {(void **)&s->rdf_nh, 8ull},
        {(void **)&H.lcell_count, 4ull * P.n_lcells}, {(void **)&H.ltmp, 4ull * P.n_lcells * P.lcapc},
        {(void **)&H.lcell, 8ull * P.n_lcells}, {(void **)&H.lid, 4ull * n}, {(void **)&H.lk, 4ull * n},
        {(void **)&H.lpos, 32ull * n}, {(void **)&H.xref, 16ull * n}, {(void **)&H.nl_n, 4ull * NL_LANES_MAX * n},
        {(void **)&H.nl, 4ull * (size_t)P.lcap * P.npad}, {(void **)&H.bslot, 4ull * NL_PART * n},
        {(void **)&H.btask, 8ull * (n / NLB_BEADS + P.n_lcells + 1)},
        {(void **)&H.tmark, 8ull * P.mark_words},
    };
    size_t total = 0;
    for (auto &it : items) total += (it.bytes + 255) / 256 * 256;
    s->arena = dalloc(s, total);
    if (!s->arena) {
        delete s;
        return fail(nullptr, MDAS_ERR_OOM, "create: device allocation of " + std::to_string(total) + " bytes failed");
    }
    s->arena_bytes = total;
    size_t off = 0;
    for (auto &it : items) {
        *it.ptr = (char *)s->arena + off;
        off += (it.bytes + 255) / 256 * 256;
    }
    H.p = dp; H.c = dc; H.n_bead_blocks = nbb;

    mdas_status st = MDAS_OK;
    {
        cudaError_t e = cudaMemsetAsync(s->arena, 0, total, s->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dp, &P, sizeof(Params), cudaMemcpyHostToDevice, s->stream);
        static const int one = 1;   // no pair list yet
        if (e == cudaSuccess) e = cudaMemcpyAsync(&dc->nl_stale, &one, sizeof(int), cudaMemcpyHostToDevice, s->stream);
        // positions: floor(x / L * 2^32) mod 2^32, with the bead's meta word
        std::vector<uint4> pos(n);
        for (int i = 0; i < n; ++i) {
            uint32_t u[3];
            for (int k = 0; k < 3; ++k) {
                const double f = std::floor(d->pos[3 * i + k] / d->box[k] * 4294967296.0);
                u[k] = (uint32_t)(uint64_t)(long long)f;
            }
            const int bt = i < nl * bpl ? d->lipid_bead_type[d->lipid_type[i / bpl] * bpl + i % bpl] : d->water_bead_type;
            const uint32_t m = i < nl * bpl ? meta_make(bt, bt, i % bpl, i / bpl + 1) : meta_make(bt, bt, 15, 0);
            pos[i] = make_uint4(u[0], u[1], u[2], m);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(H.pos, pos.data(), 16ull * n, cudaMemcpyHostToDevice, s->stream);
        if (d->precision == MDAS_FP64) {
            std::vector<Dbl4> v(n);
            for (int i = 0; i < n; ++i)
                v[i] = d->vel ? Dbl4{d->vel[3 * i], d->vel[3 * i + 1], d->vel[3 * i + 2], 0.0} : Dbl4{0.0, 0.0, 0.0, 0.0};
            if (e == cudaSuccess) e = cudaMemcpyAsync(H.vel, v.data(), 32ull * n, cudaMemcpyHostToDevice, s->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        } else {
            std::vector<float4> v(n);
            for (int i = 0; i < n; ++i)
                v[i] = d->vel ? make_float4((float)d->vel[3 * i], (float)d->vel[3 * i + 1], (float)d->vel[3 * i + 2], 0.f)
                              : make_float4(0, 0, 0, 0);
            if (e == cudaSuccess) e = cudaMemcpyAsync(H.vel, v.data(), 16ull * n, cudaMemcpyHostToDevice, s->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        }
        if (e == cudaSuccess && nl > 0) e = cudaMemcpy(H.ltype, d->lipid_type, 4ull * nl, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) st = cuda_fail(s, e, "create: upload");
    }
    if (st == MDAS_OK) st = make_batch({s}, s->solo);
    if (st == MDAS_OK) {
        cudaError_t e = cudaStreamSynchronize(s->stream);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(s, e, "create: upload");
    }
    if (st != MDAS_OK) {
        g_last_error = s->err;
        mdas_destroy_system(s);
        return st;
    }
    *out = s;
    return MDAS_OK;
}

void mdas_destroy_system(mdas_system *s) {
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    for (auto it = g_batches.begin(); it != g_batches.end();) {
        if (std::find(it->first.begin(), it->first.end(), s) != it->first.end()) {
            destroy_batch(it->second.get());
            it = g_batches.erase(it);
        } else {
            ++it;
        }
    }
    if (s->solo) destroy_batch(s->solo.get());
    dfree(s, s->arena);
    delete s;
}

mdas_status mdas_forces(mdas_system *s, double *f_out, double *u_out) {
    if (!s) return fail(nullptr, MDAS_ERR_INVALID_ARG, "forces: NULL system");
    Batch &b = *s->solo;
    LaunchCtx L = b.ctx();
    if (f_out) {
        mdas_status st = build_cells(s, b);
        if (st != MDAS_OK) return st;
        launch_pair(L, false, false, s->precision == 1);
        launch_total_force(L, s->fout, 0);
        CK(cudaMemcpyAsync(f_out, s->fout, 24ull * s->n, cudaMemcpyDeviceToHost, s->stream));
    }
    if (u_out) {
        mdas_energy_terms t;
        mdas_status st = mdas_energy(s, &t);
        if (st != MDAS_OK) return st;
        *u_out = t.potential;
    }
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaGetLastError());
    return check_err(s, b);
}

mdas_status mdas_energy(mdas_system *s, mdas_energy_terms *out) {
    if (!s || !out) return fail(s, MDAS_ERR_INVALID_ARG, "energy: NULL argument");
    Batch &b = *s->solo;
    LaunchCtx L = b.ctx();
    mdas_status st0 = build_cells(s, b);
    if (st0 != MDAS_OK) return st0;
    launch_pair(L, false, true, true);
    launch_energy_reduce(L);
    double r[8];
    CK(cudaMemcpyAsync(r, s->hs.result, sizeof(r), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaGetLastError());
    out->lj = r[0]; out->rf = r[1]; out->bond = r[2]; out->angle = r[3]; out->kinetic = r[4];
    out->pairs = (int64_t)llround(r[5]);
    out->potential = r[0] + r[1] + r[2] + r[3];
    out->total = out->potential + out->kinetic;
    return check_err(s, b);
}

mdas_status mdas_md_steps(mdas_system *s, int64_t n_steps, int32_t swap_every) {
    if (!s || n_steps < 0 || swap_every < 0) return fail(s, MDAS_ERR_INVALID_ARG, "md_steps: bad argument");
    if (s->unstable) return fail(s, MDAS_ERR_UNSTABLE, "md_steps: system is unstable; install a state first");
    return run_md(s, *s->solo, n_steps, swap_every);
}

mdas_status mdas_swap_trials(mdas_system *s, int32_t n_trials, mdas_swap_stats *stats, mdas_trial_record *log) {
    if (!s || n_trials < 0) return fail(s, MDAS_ERR_INVALID_ARG, "swap_trials: bad argument");
    if (s->unstable) return fail(s, MDAS_ERR_UNSTABLE, "swap_trials: system is unstable");
    if (n_trials == 0 || s->n_lip == 0) return MDAS_OK;
    Counters c0;
    CK(cudaMemcpyAsync(&c0, s->hs.c, sizeof(Counters), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    int rounds = 0;
    mdas_status st = run_trials(s, *s->solo, n_trials, &rounds);
    if (st != MDAS_OK) return st;
    Counters c1;
    CK(cudaMemcpyAsync(&c1, s->hs.c, sizeof(Counters), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (stats) {
        stats->trials = (int64_t)(c1.trials - c0.trials);
        stats->null_trials = (int64_t)(c1.null_trials - c0.null_trials);
        stats->accepted = (int64_t)(c1.accepted - c0.accepted);
        stats->rounds = rounds;
    }
    if (log) return mdas_trial_log(s, c0.trial, n_trials, log);
    return MDAS_OK;
}

mdas_status mdas_mutation_trials(mdas_system *s, int32_t n_trials, const double *mu, mdas_swap_stats *stats,
                                 mdas_trial_record *log) {
    if (!s || n_trials < 0) return fail(s, MDAS_ERR_INVALID_ARG, "mutation_trials: bad argument");
    double m[MAXT] = {0.0};
    if (mu)
        for (int t = 0; t < s->hp.n_lt; ++t) {
            if (!std::isfinite(mu[t])) return fail(s, MDAS_ERR_INVALID_ARG, "mutation_trials: mu is not finite");
            m[t] = mu[t];
        }
    if (s->unstable) return fail(s, MDAS_ERR_UNSTABLE, "mutation_trials: system is unstable");
    if (n_trials == 0 || s->n_lip == 0) return MDAS_OK;
    Counters c0;
    CK(cudaMemcpyAsync(&c0, s->hs.c, sizeof(Counters), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(s->hs.c->mu, m, sizeof(m), cudaMemcpyHostToDevice, s->stream));
    Batch &b = *s->solo;
    mdas_status st = build_cells(s, b);
    if (st != MDAS_OK) return st;
    LaunchCtx L = b.ctx();
    launch_mutation_trials(L, n_trials);
    s->kernel_launches += 1;
    Counters c1;
    CK(cudaMemcpyAsync(&c1, s->hs.c, sizeof(Counters), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaGetLastError());
    if (stats) {
        stats->trials = (int64_t)(c1.trials - c0.trials);
        stats->null_trials = (int64_t)(c1.null_trials - c0.null_trials);
        stats->accepted = (int64_t)(c1.accepted - c0.accepted);
        stats->rounds = 1;
    }
    st = check_err(s, b);
    if (st != MDAS_OK) return st;
    if (log) return mdas_trial_log(s, c0.trial, n_trials, log);
    return MDAS_OK;
}

mdas_status mdas_trial_log(mdas_system *s, uint64_t first, int32_t n, mdas_trial_record *rec) {
    if (!s || n < 0 || (n > 0 && !rec)) return fail(s, MDAS_ERR_INVALID_ARG, "trial_log: bad argument");
    Counters c;
    CK(cudaMemcpyAsync(&c, s->hs.c, sizeof(Counters), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (first + (uint64_t)n > c.trial || c.trial - first > (uint64_t)LOG_CAP)
        return fail(s, MDAS_ERR_INVALID_ARG, "trial_log: records not in the log");
    static_assert(sizeof(TrialRec) == sizeof(mdas_trial_record), "trial record layout");
    for (int k = 0; k < n;) {
        const uint64_t idx = (first + k) % LOG_CAP;
        const int m = (int)std::min<uint64_t>((uint64_t)(n - k), LOG_CAP - idx);
        CK(cudaMemcpyAsync(rec + k, s->hs.log + idx, sizeof(TrialRec) * m, cudaMemcpyDeviceToHost, s->stream));
        k += m;
    }
    CK(cudaStreamSynchronize(s->stream));
    return MDAS_OK;
}

}  // extern "C"

namespace {

// Per-block output of a traced alchemical move (host arrays, any may be NULL).
struct MoveTrace {
    double *w;          // [n_lambda] work added by each block
    uint32_t *pos;      // [n_lambda][n][3] fixed-point positions after each block
    double *vel;        // [n_lambda][n][3] velocities after each block
};

// After lambda block k (0-based) of a traced move: the work the block added
// (the running work minus *w_prev), the positions and the velocities.
mdas_status trace_block(mdas_system *s, int k, double *w_prev, const MoveTrace &tr) {
    const size_t n = (size_t)s->n;
    double w = 0.0;
    CK(cudaMemcpyAsync(&w, &s->hs.c->w, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    std::vector<uint4> p(tr.pos ? n : 0);
    if (tr.pos) CK(cudaMemcpyAsync(p.data(), s->hs.pos, 16 * n, cudaMemcpyDeviceToHost, s->stream));
    std::vector<Dbl4> vd(tr.vel && s->precision == 1 ? n : 0);
    std::vector<float4> vf(tr.vel && s->precision != 1 ? n : 0);
    if (tr.vel && s->precision == 1) CK(cudaMemcpyAsync(vd.data(), s->hs.vel, 32 * n, cudaMemcpyDeviceToHost, s->stream));
    if (tr.vel && s->precision != 1) CK(cudaMemcpyAsync(vf.data(), s->hs.vel, 16 * n, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (tr.w) tr.w[k] = w - *w_prev;
    *w_prev = w;
    for (size_t i = 0; tr.pos && i < n; ++i) {
        uint32_t *o = tr.pos + ((size_t)k * n + i) * 3;
        o[0] = p[i].x; o[1] = p[i].y; o[2] = p[i].z;
    }
    for (size_t i = 0; tr.vel && i < n; ++i) {
        double *o = tr.vel + ((size_t)k * n + i) * 3;
        if (s->precision == 1) { o[0] = vd[i].x; o[1] = vd[i].y; o[2] = vd[i].z; }
        else { o[0] = vf[i].x; o[1] = vf[i].y; o[2] = vf[i].z; }
    }
    return MDAS_OK;
}

// One MDAS move (Sec. 2, Eqs. 2-3) with pairs given (pairs), drawn over all
// lipids (mode 0) or drawn across the leaflets (mode 2, head_k).  With a
// trace, the trajectory runs one lambda block per MD run (the bits of one
// run) and each block's work, positions and velocities are copied out.
mdas_status alchemical_move(mdas_system *s, int32_t n_pairs, int32_t n_lambda, int32_t md_per_lambda,
                            const int32_t *pairs, int mode, int head_k, mdas_move_result *res, const MoveTrace *tr) {
    if (!s || n_pairs < 0 || n_pairs > MAX_PAIRS || n_lambda < 1 || md_per_lambda < 0)
        return fail(s, MDAS_ERR_INVALID_ARG, "alchemical_move: bad argument");
    if (s->unstable) return fail(s, MDAS_ERR_UNSTABLE, "alchemical_move: system is unstable");
    Batch &b = *s->solo;
    LaunchCtx L = b.ctx();
    if (pairs) {
        std::vector<int> lt(std::max(s->n_lip, 1));
        CK(cudaMemcpy(lt.data(), s->hs.ltype, 4ull * s->n_lip, cudaMemcpyDeviceToHost));
        std::vector<char> used(s->n_lip, 0);
        for (int p = 0; p < 2 * n_pairs; ++p) {
            const int l = pairs[p];
            if (l < 0 || l >= s->n_lip || used[l]) return fail(s, MDAS_ERR_INVALID_ARG, "alchemical_move: pairs must be distinct lipids");
            used[l] = 1;
        }
        for (int p = 0; p < n_pairs; ++p)
            if (lt[pairs[2 * p]] == lt[pairs[2 * p + 1]]) return fail(s, MDAS_ERR_INVALID_ARG, "alchemical_move: a pair shares its type");
        Counters *dc = s->hs.c;
        CK(cudaMemcpyAsync(&dc->pairs, pairs, 8ull * n_pairs, cudaMemcpyHostToDevice, s->stream));
        CK(cudaMemcpyAsync(&dc->n_pairs, &n_pairs, 4, cudaMemcpyHostToDevice, s->stream));
        mode = 1;
    }
    int *leaf = nullptr;
    if (mode == 2) {
        // leaflets at the start of the move (scratch: the head-bead info array)
        leaf = reinterpret_cast<int *>(s->rdf_info);
        launch_leaflets(L, s->n_lip, head_k, leaf);
    }
    launch_snapshot(L);
    launch_mdas_select(L, n_pairs, 64 * n_pairs + 64, mode, leaf);
    int np = 0;
    CK(cudaMemcpyAsync(&np, &s->hs.c->n_pairs, 4, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (np > 0) {
        const double dl = 1.0 / n_lambda;
        double w_prev = 0.0;
        if (md_per_lambda > 0) {
            // the whole trajectory in one MD run: lambda advances by dl after
            // every md_per_lambda steps, each block's work term from the pair
            // list (valid right after the block's steps)
            launch_mdas_set_lambda(L, 0.0, 1);
            if (!tr) {
                mdas_status st = run_md(s, b, (long long)n_lambda * md_per_lambda, 0, true, false, md_per_lambda, dl);
                if (st != MDAS_OK) return st;
            } else {
                for (int k = 0; k < n_lambda; ++k) {
                    mdas_status st = run_md(s, b, md_per_lambda, 0, true, false, md_per_lambda, dl,
                                            (long long)k * md_per_lambda);
                    if (st == MDAS_OK) st = trace_block(s, k, &w_prev, *tr);
                    if (st != MDAS_OK) return st;
                }
            }
        } else {
            for (int k = 1; k <= n_lambda; ++k) {
                launch_mdas_set_lambda(L, (double)(k - 1) / n_lambda, 1);
                mdas_status st = build_cells(s, b);
                if (st != MDAS_OK) return st;
                launch_mdas_dE(L, dl);
                if (tr && (st = trace_block(s, k - 1, &w_prev, *tr)) != MDAS_OK) return st;
            }
        }
    }
    launch_mdas_accept(L);
    launch_mdas_restore(L);
    s->cells_valid = false;
    Counters c;
    double r[10];
    CK(cudaMemcpyAsync(&c, s->hs.c, sizeof(Counters), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(r, s->hs.result, sizeof(r), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaGetLastError());
    if (res) {
        res->w = c.w;
        res->u = r[9];
        res->accepted = c.mdas_accept;
        res->n_pairs = c.n_pairs;
        for (int k = 0; k < 2 * c.n_pairs; ++k) res->pairs[k] = c.pairs[k];
    }
    return check_err(s, b);
}

}  // namespace

extern "C" {

mdas_status mdas_alchemical_move(mdas_system *s, int32_t n_pairs, int32_t n_lambda, int32_t md_per_lambda,
                                 const int32_t *pairs, mdas_move_result *res) {
    return alchemical_move(s, n_pairs, n_lambda, md_per_lambda, pairs, 0, 1, res, nullptr);
}

mdas_status mdas_alchemical_move_trace(mdas_system *s, int32_t n_pairs, int32_t n_lambda, int32_t md_per_lambda,
                                       const int32_t *pairs, mdas_move_result *res, double *w_blocks,
                                       uint32_t *pos_blocks, double *vel_blocks) {
    const MoveTrace tr{w_blocks, pos_blocks, vel_blocks};
    return alchemical_move(s, n_pairs, n_lambda, md_per_lambda, pairs, 0, 1, res, &tr);
}

mdas_status mdas_interleaflet_move(mdas_system *s, int32_t n_pairs, int32_t n_lambda, int32_t md_per_lambda,
                                   int32_t head_k, mdas_move_result *res) {
    if (s && (head_k < 0 || head_k >= s->bpl - 1))
        return fail(s, MDAS_ERR_INVALID_ARG, "interleaflet_move: head_k outside [0, beads_per_lipid - 1)");
    return alchemical_move(s, n_pairs, n_lambda, md_per_lambda, nullptr, 2, head_k, res, nullptr);
}

mdas_status mdas_device_ptrs(mdas_system *s, mdas_device_view *out) {
    if (!s || !out) return fail(s, MDAS_ERR_INVALID_ARG, "device_ptrs: NULL argument");
    out->pos = s->hs.pos;
    out->vel = s->hs.vel;
    out->lipid_type = s->hs.ltype;
    out->n_beads = s->n;
    out->n_lipids = s->n_lip;
    out->precision = s->precision;
    out->vel_stride_bytes = s->precision == 1 ? 32 : 16;
    for (int k = 0; k < 3; ++k) out->box[k] = s->hp.box[k];
    return MDAS_OK;
}

mdas_status mdas_delta_energy(mdas_system *s, const int32_t *lipids, const int32_t *new_types, int32_t n, double *dE) {
    if (!s || !dE || n < 0 || n > MAX_PAIRS || (n > 0 && (!lipids || !new_types)))
        return fail(s, MDAS_ERR_INVALID_ARG, "delta_energy: bad argument (at most 64 lipids)");
    for (int k = 0; k < n; ++k) {
        if (lipids[k] < 0 || lipids[k] >= s->n_lip || new_types[k] < 0 || new_types[k] >= s->hp.n_lt)
            return fail(s, MDAS_ERR_INVALID_ARG, "delta_energy: lipid or type out of range");
        for (int j = 0; j < k; ++j)
            if (lipids[j] == lipids[k]) return fail(s, MDAS_ERR_INVALID_ARG, "delta_energy: lipids must be distinct");
    }
    if (n == 0) { *dE = 0.0; return MDAS_OK; }
    Batch &b = *s->solo;
    LaunchCtx L = b.ctx();
    Counters *dc = s->hs.c;
    int np_save = 0;
    CK(cudaMemcpyAsync(&np_save, &dc->n_pairs, 4, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(&dc->pairs[0], lipids, 4ull * n, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(&dc->pairs[MAX_PAIRS], new_types, 4ull * n, cudaMemcpyHostToDevice, s->stream));
    mdas_status st0 = build_cells(s, b);
    if (st0 != MDAS_OK) return st0;
    launch_delta_energy(L, n);
    CK(cudaMemcpyAsync(dE, s->hs.result + 8, 8, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaMemcpyAsync(&dc->n_pairs, &np_save, 4, cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaGetLastError());
    return MDAS_OK;
}

mdas_status mdas_get_state(const mdas_system *cs, mdas_state_view *out) {
    mdas_system *s = const_cast<mdas_system *>(cs);
    if (!s || !out) return fail(s, MDAS_ERR_INVALID_ARG, "get_state: NULL argument");
    const int n = s->n;
    std::vector<uint4> pos(n);
    CK(cudaMemcpyAsync(pos.data(), s->hs.pos, 16ull * n, cudaMemcpyDeviceToHost, s->stream));
    Counters c;
    CK(cudaMemcpyAsync(&c, s->hs.c, sizeof(c), cudaMemcpyDeviceToHost, s->stream));
    std::vector<double> v(3ull * n);
    if (out->vel) {
        if (s->precision == MDAS_FP64) {
            std::vector<Dbl4> dv(n);
            CK(cudaMemcpyAsync(dv.data(), s->hs.vel, 32ull * n, cudaMemcpyDeviceToHost, s->stream));
            CK(cudaStreamSynchronize(s->stream));
            for (int i = 0; i < n; ++i) { out->vel[3 * i] = dv[i].x; out->vel[3 * i + 1] = dv[i].y; out->vel[3 * i + 2] = dv[i].z; }
        } else {
            std::vector<float4> fv(n);
            CK(cudaMemcpyAsync(fv.data(), s->hs.vel, 16ull * n, cudaMemcpyDeviceToHost, s->stream));
            CK(cudaStreamSynchronize(s->stream));
            for (int i = 0; i < n; ++i) { out->vel[3 * i] = fv[i].x; out->vel[3 * i + 1] = fv[i].y; out->vel[3 * i + 2] = fv[i].z; }
        }
    }
    if (out->lipid_type && s->n_lip > 0)
        CK(cudaMemcpyAsync(out->lipid_type, s->hs.ltype, 4ull * s->n_lip, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    for (int i = 0; i < n; ++i) {
        const uint32_t u[3] = {pos[i].x, pos[i].y, pos[i].z};
        for (int k = 0; k < 3; ++k) {
            if (out->pos_fixed) out->pos_fixed[3 * i + k] = u[k];
            if (out->pos) out->pos[3 * i + k] = (double)u[k] * s->hp.qs[k];
        }
    }
    out->step = c.step; out->trial = c.trial; out->move = c.move; out->at_step = c.at_step;
    // the continuation state: the positions the pair list was built at (kept
    // in list order on the device) and the kinetic energy of the last step
    out->list_valid = 0;
    if (out->list_ref && !c.nl_stale && !c.nl_viol) {
        std::vector<uint4> xr(n);
        std::vector<int> lk(n);
        CK(cudaMemcpyAsync(xr.data(), s->hs.xref, 16ull * n, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaMemcpyAsync(lk.data(), s->hs.lk, 4ull * n, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        for (int i = 0; i < n; ++i) {
            const uint4 r = xr[lk[i]];
            out->list_ref[3 * i] = r.x; out->list_ref[3 * i + 1] = r.y; out->list_ref[3 * i + 2] = r.z;
        }
        out->list_valid = 1;
    }
    out->ke_valid = c.ke_fresh;
    out->ke[0] = c.ke_fresh ? c.ke_total[0] : 0.0;
    out->ke[1] = c.ke_fresh ? c.ke_total[1] : 0.0;
    for (int k = 0; k < 3; ++k) {
        out->box[k] = s->hp.box[k];
        out->box_velocity[k] = s->hp.boxv[k];
        out->list_box[k] = out->list_valid ? c.lbox[k] : 0.0;
    }
    return MDAS_OK;
}

mdas_status mdas_box(const mdas_system *s, double box[3], double box_velocity[3], double pressure[3]) {
    if (!s) return fail(nullptr, MDAS_ERR_INVALID_ARG, "box: NULL system");
    for (int k = 0; k < 3; ++k) {
        if (box) box[k] = s->hp.box[k];
        if (box_velocity) box_velocity[k] = s->hp.boxv[k];
        if (pressure) pressure[k] = s->hp.pres[k];
    }
    return MDAS_OK;
}

mdas_status mdas_wait_timeout_probe(mdas_system *s) {
    if (!s) return fail(nullptr, MDAS_ERR_INVALID_ARG, "wait_timeout_probe: NULL system");
    Batch &b = *s->solo;
    CK(launch_barrier_stall(b.rsync, b.stream));
    k_run_abort<<<1, 32, 0, b.stream>>>(b.rsync, (int)md_run_sync_bytes(), b.dsys, (int)b.sys.size(), nullptr);
    CK(cudaGetLastError());
    return check_err(s, b);
}

// After a list build at the saved build positions: the current positions
// (id order) into the list-order buffer the next step reads.
__global__ void k_list_current(const SysDev S, int n, int par) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    S.lpos[(size_t)par * n + k] = S.pos[S.lid[k]];
}

// The counters of a newly installed state (both ways of installing one):
// no error, no pending exchange, alchemical or kinetic-energy work, the pair
// list to be rebuilt.  The step, trial and move counters are the caller's.
__host__ __device__ inline void new_state_counters(Counters &c) {
    c.err = 0; c.in_at = 0; c.lambda = 0.0; c.pending = 0; c.ke_fresh = 0; c.ke_pending = 0; c.draw_n = 0;
    for (int g = 0; g < 2; ++g)
        for (int q = 0; q < KE_SLOTS; ++q) c.ke_slot[g][q][0] = c.ke_slot[g][q][1] = 0;
    c.nl_stale = 1; c.nl_viol = 0; c.sticket = 0; c.nticket = 0;
}

// A packed state upload, after the copies: each bead's meta word from the
// lipid types (the host checked them), the counters of a new state.
__global__ void k_state_packed(const SysDev S, int n, int nl, int bpl, int water_bt) {
    const Params &P = *S.p;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        uint4 q = S.pos[i];
        if (i < nl * bpl) {
            const int bt = P.lbt[S.ltype[i / bpl] * 16 + i % bpl];
            q.w = meta_make(bt, bt, i % bpl, i / bpl + 1);
        } else {
            q.w = meta_make(water_bt, water_bt, 15, 0);
        }
        S.pos[i] = q;
    }
    if (i == 0) new_state_counters(*S.c);
}

mdas_status mdas_get_state_packed(const mdas_system *cs, uint32_t *pos4, void *vel4, int32_t *lipid_type) {
    mdas_system *s = const_cast<mdas_system *>(cs);
    if (!s) return fail(nullptr, MDAS_ERR_INVALID_ARG, "get_state_packed: NULL system");
    const size_t n = s->n, vsz = s->precision == MDAS_FP64 ? 32 : 16;
    if (pos4) CK(cudaMemcpyAsync(pos4, s->hs.pos, 16 * n, cudaMemcpyDeviceToHost, s->stream));
    if (vel4) CK(cudaMemcpyAsync(vel4, s->hs.vel, vsz * n, cudaMemcpyDeviceToHost, s->stream));
    if (lipid_type && s->n_lip > 0)
        CK(cudaMemcpyAsync(lipid_type, s->hs.ltype, 4ull * s->n_lip, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return MDAS_OK;
}

mdas_status mdas_set_state_packed(mdas_system *s, const uint32_t *pos4, const void *vel4, const int32_t *lipid_type) {
    if (!s) return fail(nullptr, MDAS_ERR_INVALID_ARG, "set_state_packed: NULL system");
    const size_t n = s->n, vsz = s->precision == MDAS_FP64 ? 32 : 16;
    if (lipid_type)
        for (int l = 0; l < s->n_lip; ++l)
            if (lipid_type[l] < 0 || lipid_type[l] >= s->hp.n_lt)
                return fail(s, MDAS_ERR_INVALID_ARG, "set_state_packed: lipid type");
    if (pos4) CK(cudaMemcpyAsync(s->hs.pos, pos4, 16 * n, cudaMemcpyHostToDevice, s->stream));
    if (vel4) CK(cudaMemcpyAsync(s->hs.vel, vel4, vsz * n, cudaMemcpyHostToDevice, s->stream));
    if (lipid_type && s->n_lip > 0)
        CK(cudaMemcpyAsync(s->hs.ltype, lipid_type, 4ull * s->n_lip, cudaMemcpyHostToDevice, s->stream));
    k_state_packed<<<(int)((n + 255) / 256), 256, 0, s->stream>>>(s->hs, (int)n, s->n_lip, s->bpl, s->water_bt);
    CK(cudaGetLastError());
    // the host arrays may be reused once the call returns
    CK(cudaStreamSynchronize(s->stream));
    s->unstable = false;
    s->cells_valid = false;
    return MDAS_OK;
}

mdas_status mdas_set_state(mdas_system *s, const mdas_state_view *in) {
    if (!s || !in) return fail(s, MDAS_ERR_INVALID_ARG, "set_state: NULL argument");
    const int n = s->n, nl = s->n_lip, bpl = s->bpl;
    const bool keep_list = in->list_valid && in->list_ref;
    if (keep_list && !in->pos_fixed && !in->pos)
        return fail(s, MDAS_ERR_INVALID_ARG, "set_state: list_ref without positions");
    if (in->box[0] > 0) {
        // a new box (pressure coupling state): first, so that positions in nm convert with it
        for (int k = 0; k < 3; ++k)
            if (!(in->box[k] >= s->hp.pc_lmin[k]) || !std::isfinite(in->box[k]) || !std::isfinite(in->box_velocity[k]))
                return fail(s, MDAS_ERR_INVALID_ARG, "set_state: box below what the cell grids allow, or not finite");
        for (int k = 0; k < 3; ++k) {
            box_params(s->hp, k, in->box[k]);
            s->hp.boxv[k] = s->hp.pc_nst > 0 ? in->box_velocity[k] : 0.0;
            s->hp.dtm_pc[k] = s->hp.dt * (s->hp.boxv[k] / in->box[k]);
            s->hp.dtm_pcf[k] = (float)s->hp.dtm_pc[k];
        }
        CK(cudaMemcpyAsync(const_cast<Params *>(s->hs.p), &s->hp, sizeof(Params), cudaMemcpyHostToDevice, s->stream));
    }
    std::vector<int> lt(std::max(nl, 1));
    if (in->lipid_type) {
        for (int l = 0; l < nl; ++l)
            if (in->lipid_type[l] < 0 || in->lipid_type[l] >= s->hp.n_lt) return fail(s, MDAS_ERR_INVALID_ARG, "set_state: lipid type");
        std::copy(in->lipid_type, in->lipid_type + nl, lt.begin());
    } else if (nl > 0) {
        CK(cudaMemcpy(lt.data(), s->hs.ltype, 4ull * nl, cudaMemcpyDeviceToHost));
    }
    std::vector<uint4> pos(n);
    if (!in->pos_fixed && !in->pos) {   // keep the current coordinates
        CK(cudaMemcpyAsync(pos.data(), s->hs.pos, 16ull * n, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    }
    for (int i = 0; i < n; ++i) {
        if (in->pos_fixed) {
            pos[i].x = in->pos_fixed[3 * i]; pos[i].y = in->pos_fixed[3 * i + 1]; pos[i].z = in->pos_fixed[3 * i + 2];
        } else if (in->pos) {
            uint32_t u[3];
            for (int k = 0; k < 3; ++k)
                u[k] = (uint32_t)(uint64_t)(long long)std::floor(in->pos[3 * i + k] / s->hp.box[k] * 4294967296.0);
            pos[i].x = u[0]; pos[i].y = u[1]; pos[i].z = u[2];
        }
        if (i < nl * bpl) {
            const int bt = s->hp.lbt[lt[i / bpl] * 16 + i % bpl];
            pos[i].w = meta_make(bt, bt, i % bpl, i / bpl + 1);
        } else {
            pos[i].w = meta_make(s->water_bt, s->water_bt, 15, 0);
        }
    }
    std::vector<uint4> ref;
    if (keep_list) {
        // every bead within half the skin of the build position (in FP64; the
        // step's own test is tighter by 1e-4 of the square)
        const double half = 0.5 * (s->hp.rl - s->hp.rc);
        ref.resize(n);
        for (int i = 0; i < n; ++i) {
            const uint32_t r[3] = {in->list_ref[3 * i], in->list_ref[3 * i + 1], in->list_ref[3 * i + 2]};
            const uint32_t u[3] = {pos[i].x, pos[i].y, pos[i].z};
            double d2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double d = (double)(int32_t)(u[k] - r[k]) * s->hp.qs[k];
                d2 += d * d;
            }
            if (!(d2 <= half * half)) return fail(s, MDAS_ERR_INVALID_ARG, "set_state: list_ref farther than half the skin");
            ref[i] = make_uint4(r[0], r[1], r[2], pos[i].w);
        }
    }
    CK(cudaMemcpyAsync(s->hs.pos, keep_list ? ref.data() : pos.data(), 16ull * n, cudaMemcpyHostToDevice, s->stream));
    if (nl > 0) CK(cudaMemcpyAsync(s->hs.ltype, lt.data(), 4ull * nl, cudaMemcpyHostToDevice, s->stream));
    if (in->vel) {
        if (s->precision == MDAS_FP64) {
            std::vector<Dbl4> v(n);
            for (int i = 0; i < n; ++i) v[i] = Dbl4{in->vel[3 * i], in->vel[3 * i + 1], in->vel[3 * i + 2], 0.0};
            CK(cudaMemcpyAsync(s->hs.vel, v.data(), 32ull * n, cudaMemcpyHostToDevice, s->stream));
            CK(cudaStreamSynchronize(s->stream));
        } else {
            std::vector<float4> v(n);
            for (int i = 0; i < n; ++i) v[i] = make_float4((float)in->vel[3 * i], (float)in->vel[3 * i + 1], (float)in->vel[3 * i + 2], 0.f);
            CK(cudaMemcpyAsync(s->hs.vel, v.data(), 16ull * n, cudaMemcpyHostToDevice, s->stream));
            CK(cudaStreamSynchronize(s->stream));
        }
    }
    Counters c;
    CK(cudaMemcpyAsync(&c, s->hs.c, sizeof(c), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    c.step = in->step; c.trial = in->trial; c.move = in->move; c.at_step = in->at_step;
    new_state_counters(c);
    if (in->ke_valid) {
        c.ke_fresh = 1;
        c.ke_total[0] = in->ke[0];
        c.ke_total[1] = in->ke[1];
    }
    if (keep_list) c.nl_par = 0;
    CK(cudaMemcpyAsync(s->hs.c, &c, sizeof(c), cudaMemcpyHostToDevice, s->stream));
    if (keep_list) {
        // the list as it was built (same positions, same order, and under
        // pressure coupling the same box: the build's distances in nm follow
        // the box), then the current positions in its list-order buffer
        bool other_box = false;
        for (int k = 0; k < 3; ++k) other_box |= in->list_box[0] > 0 && in->list_box[k] != s->hp.box[k];
        Params lp = s->hp;
        if (other_box) {
            for (int k = 0; k < 3; ++k) {
                if (!(in->list_box[k] >= s->hp.pc_lmin[k]) || !std::isfinite(in->list_box[k]))
                    return fail(s, MDAS_ERR_INVALID_ARG, "set_state: list_box");
                box_params(lp, k, in->list_box[k]);
            }
            CK(cudaMemcpyAsync(const_cast<Params *>(s->hs.p), &lp, sizeof(Params), cudaMemcpyHostToDevice, s->stream));
        }
        launch_nl_build(s->solo->ctx());
        if (other_box)
            CK(cudaMemcpyAsync(const_cast<Params *>(s->hs.p), &s->hp, sizeof(Params), cudaMemcpyHostToDevice, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        s->list_lanes = s->solo->lanes;
        CK(cudaMemcpyAsync(s->hs.pos, pos.data(), 16ull * n, cudaMemcpyHostToDevice, s->stream));
        k_list_current<<<(n + 255) / 256, 256, 0, s->stream>>>(s->hs, n, 0);
        if (in->list_box[0] > 0) {
            // the box the saved list was built at, and the displacement bound that follows
            double mu = 1.0;
            for (int k = 0; k < 3; ++k) {
                if (!(in->list_box[k] > 0) || !std::isfinite(in->list_box[k]))
                    return fail(s, MDAS_ERR_INVALID_ARG, "set_state: list_box");
                mu = std::min(mu, s->hp.box[k] / in->list_box[k]);
            }
            double lb[3];
            for (int k = 0; k < 3; ++k) lb[k] = in->list_box[k];
            const float d2 = mu * s->hp.rl - s->hp.rc > 0.0 ? list_dmax2f(s->hp.rl, s->hp.rc, mu) : 0.0f;
            CK(cudaMemcpyAsync(s->hs.c->lbox, lb, sizeof(lb), cudaMemcpyHostToDevice, s->stream));
            CK(cudaMemcpyAsync(&s->hs.c->dmax2f, &d2, sizeof(d2), cudaMemcpyHostToDevice, s->stream));
            CK(cudaStreamSynchronize(s->stream));
        }
    }
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaGetLastError());
    s->unstable = false;
    s->cells_valid = false;
    return MDAS_OK;
}

mdas_status mdas_cell_list(mdas_system *s, int32_t *sorted_ids, int32_t *cell_start, int32_t *ncell) {
    if (!s) return fail(nullptr, MDAS_ERR_INVALID_ARG, "cell_list: NULL system");
    mdas_status st0 = build_cells(s, *s->solo);
    if (st0 != MDAS_OK) return st0;
    const int nc = s->hp.n_cells, capc = s->hp.capc;
    std::vector<int> cnt(nc), ids((size_t)nc * capc);
    CK(cudaMemcpyAsync(cnt.data(), s->hs.cell_n, 4ull * nc, cudaMemcpyDeviceToHost, s->stream));
    if (sorted_ids) CK(cudaMemcpyAsync(ids.data(), s->hs.sorted_id, 4ull * nc * capc, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaGetLastError());
    int o = 0;
    for (int c = 0; c < nc; ++c) {
        if (cell_start) cell_start[c] = o;
        if (sorted_ids)
            for (int k = 0; k < cnt[c]; ++k) sorted_ids[o + k] = ids[(size_t)c * capc + k];
        o += cnt[c];
    }
    if (cell_start) cell_start[nc] = o;
    if (ncell) for (int k = 0; k < 3; ++k) ncell[k] = s->hp.nc[k];
    if (o != s->n) return fail(s, MDAS_ERR_UNSTABLE, "cell_list: a cell overflowed its capacity");
    return check_err(s, *s->solo);
}

mdas_status mdas_batch_run(mdas_system *const *systems, int32_t n_systems, int32_t md_steps, int32_t swap_trials) {
    if (!systems || n_systems <= 0 || md_steps < 0 || swap_trials < 0)
        return fail(nullptr, MDAS_ERR_INVALID_ARG, "batch_run: bad argument");
    std::vector<mdas_system *> v(systems, systems + n_systems);
    for (auto *x : v) {
        if (!x) return fail(nullptr, MDAS_ERR_INVALID_ARG, "batch_run: NULL system");
        if (x->unstable) return fail(x, MDAS_ERR_UNSTABLE, "batch_run: a system is unstable");
    }
    mdas_system *s = v[0];
    auto batch_of = [&](const std::vector<mdas_system *> &w, Batch **out) {
        auto it = g_batches.find(w);
        if (it == g_batches.end()) {
            std::unique_ptr<Batch> b;
            mdas_status st = make_batch(w, b);
            if (st != MDAS_OK) return st;
            it = g_batches.emplace(w, std::move(b)).first;
        } else {
            // a system changed its step shape since the batch was made: the
            // batch's step items follow (and the systems must still agree)
            bool same = true;
            for (auto *x : w) same = same && x->lanes == it->second->lanes;
            if (!same) {
                mdas_status st = refill_batch(*it->second, w);
                if (st != MDAS_OK) return st;
            }
        }
        *out = it->second.get();
        return MDAS_OK;
    };
    Batch *bp = nullptr;
    mdas_status st = batch_of(v, &bp);
    if (st != MDAS_OK) return st;
    Batch &b = *bp;
    long long total = 0;
    for (auto *x : v) total += x->n;
    const long long wave = s->wave_beads;
    if (wave > 0 && total > wave && md_steps > 0) {
        // MD in waves of consecutive systems (each wave's working set closer
        // to what the L2 cache holds); every system's arithmetic is its own,
        // so the bits are those of one batch
        for (size_t k = 0; k < v.size();) {
            std::vector<mdas_system *> w;
            long long beads = 0;
            while (k < v.size() && (w.empty() || beads + v[k]->n <= wave)) { beads += v[k]->n; w.push_back(v[k++]); }
            Batch *wb = nullptr;
            st = batch_of(w, &wb);
            if (st == MDAS_OK) st = run_md(w[0], *wb, md_steps, 0);
            if (st != MDAS_OK) return st;
        }
    } else {
        st = run_md(s, b, md_steps, 0);
        if (st != MDAS_OK) return st;
    }
    if (swap_trials > 0) {
        for (auto *x : v)
            if (x->n_lip == 0) return fail(x, MDAS_ERR_INVALID_ARG, "batch_run: a system has no lipids");
        st = run_trials(s, b, swap_trials, nullptr);
    }
    return st;
}

mdas_status mdas_head_rdf(mdas_system *s, int32_t lipid_type, int32_t head_k, double r_max, int32_t n_bins,
                          int64_t *counts_out, int32_t *n_heads_out) {
    if (!s || !counts_out || !n_heads_out) return fail(s, MDAS_ERR_INVALID_ARG, "head_rdf: NULL argument");
    if (lipid_type < 0 || lipid_type >= s->hp.n_lt || head_k < 0 || head_k >= s->bpl - 1)
        return fail(s, MDAS_ERR_INVALID_ARG, "head_rdf: lipid type or head bead out of range");
    if (n_bins < 1 || n_bins > RDF_MAX_BINS || !(r_max > 0.0) ||
        r_max > 0.5 * std::min(s->hp.box[0], s->hp.box[1]))
        return fail(s, MDAS_ERR_INVALID_ARG, "head_rdf: n_bins outside [1, 1024] or r_max outside (0, L/2]");
    if (s->unstable) return fail(s, MDAS_ERR_UNSTABLE, "head_rdf: the system is unstable");
    Batch &b = *s->solo;
    LaunchCtx L = b.ctx();
    launch_head_rdf(L.sys, s->n_lip, lipid_type, head_k, r_max, n_bins, s->rdf_info, s->rdf_nh, s->rdf_hist,
                    s->stream);
    std::vector<unsigned long long> h(2 * (size_t)n_bins);
    int nh[2];
    CK(cudaMemcpyAsync(h.data(), s->rdf_hist, 8ull * 2 * n_bins, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(nh, s->rdf_nh, 8, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaGetLastError());
    for (int k = 0; k < 2 * n_bins; ++k) counts_out[k] = (int64_t)h[k];
    n_heads_out[0] = nh[0];
    n_heads_out[1] = nh[1];
    return MDAS_OK;
}

}  // extern "C"

namespace {

// Device time per MD step of a batch made from descs with the given list
// skin, layout (partitioned or in lockstep), wave size and list columns per
// bead: one untimed round, then `rounds` rounds of mdas_batch_run timed with
// CUDA events on the batch's stream; the systems are destroyed afterwards.
mdas_status time_batch(const mdas_system_desc *const *descs, int n_systems, double skin, int partitioned,
                       long long wave, int lanes, int md_steps, int swap_trials, int rounds, double *us) {
    std::vector<mdas_system_desc> dv(n_systems);
    std::vector<mdas_system *> sv;
    for (int i = 0; i < n_systems; ++i) {
        dv[i] = *descs[i];
        dv[i].list_skin = skin;
    }
    mdas_status st = MDAS_OK;
    for (int i = 0; i < n_systems && st == MDAS_OK; ++i) {
        mdas_system *x = nullptr;
        st = mdas_create_system(&dv[i], &x);
        if (st == MDAS_OK) {
            x->partition = partitioned != 0;
            x->wave_beads = wave;
            sv.push_back(x);
            st = mdas_set_list_lanes(x, lanes);
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    if (st == MDAS_OK) st = mdas_batch_run(sv.data(), n_systems, md_steps, swap_trials);   // untimed round
    if (st == MDAS_OK) {
        cudaStream_t q = sv[0]->stream;
        cudaError_t e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e == cudaSuccess) e = cudaEventRecord(e0, q);
        for (int r = 0; r < rounds && e == cudaSuccess && st == MDAS_OK; ++r)
            st = mdas_batch_run(sv.data(), n_systems, md_steps, swap_trials);
        if (e == cudaSuccess && st == MDAS_OK) e = cudaEventRecord(e1, q);
        if (e == cudaSuccess && st == MDAS_OK) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess && st == MDAS_OK) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess && st == MDAS_OK) st = cuda_fail(nullptr, e, "tune: timing");
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (auto *x : sv) mdas_destroy_system(x);
    if (st == MDAS_OK) *us = 1e3 * (double)ms / ((double)rounds * md_steps);
    return st;
}

mdas_status tune_args(const char *who, const mdas_system_desc *const *descs, int32_t n_systems, const double *skins,
                      int32_t n_skins, int32_t md_steps, int32_t swap_trials, int32_t rounds) {
    if (!descs || n_systems <= 0 || !skins || n_skins <= 0 || md_steps <= 0 || swap_trials < 0 || rounds <= 0)
        return fail(nullptr, MDAS_ERR_INVALID_ARG, std::string(who) + ": bad argument");
    for (int i = 0; i < n_systems; ++i)
        if (!descs[i]) return fail(nullptr, MDAS_ERR_INVALID_ARG, std::string(who) + ": NULL descriptor");
    for (int c = 0; c < n_skins; ++c)
        if (!(skins[c] > 0.0)) return fail(nullptr, MDAS_ERR_INVALID_ARG, std::string(who) + ": a candidate skin is <= 0");
    return MDAS_OK;
}

}  // namespace

extern "C" {

mdas_status mdas_tune_list_skin(const mdas_system_desc *const *descs, int32_t n_systems, const double *skins,
                                int32_t n_skins, int32_t md_steps, int32_t swap_trials, int32_t rounds,
                                double *us_per_step, double *best_skin) {
    mdas_status st = tune_args("tune_list_skin", descs, n_systems, skins, n_skins, md_steps, swap_trials, rounds);
    if (st != MDAS_OK) return st;
    if (!us_per_step || !best_skin) return fail(nullptr, MDAS_ERR_INVALID_ARG, "tune_list_skin: bad argument");
    int best = -1;
    for (int c = 0; c < n_skins; ++c) {
        st = time_batch(descs, n_systems, skins[c], 1, 0, NL_LANES, md_steps, swap_trials, rounds, &us_per_step[c]);
        if (st != MDAS_OK) return st;
        if (best < 0 || us_per_step[c] < us_per_step[best]) best = c;
    }
    *best_skin = skins[best];
    return MDAS_OK;
}

mdas_status mdas_tune_batch(const mdas_system_desc *const *descs, int32_t n_systems, const double *skins,
                            int32_t n_skins, const int64_t *waves, int32_t n_waves, const int32_t *lanes,
                            int32_t n_lanes, int32_t md_steps, int32_t swap_trials, int32_t rounds,
                            double *us_per_step, double *best_skin, int32_t *best_partitioned, int64_t *best_wave,
                            int32_t *best_lanes) {
    mdas_status st = tune_args("tune_batch", descs, n_systems, skins, n_skins, md_steps, swap_trials, rounds);
    if (st != MDAS_OK) return st;
    if (!waves || n_waves <= 0 || !lanes || n_lanes <= 0 || !us_per_step || !best_skin || !best_partitioned ||
        !best_wave || !best_lanes)
        return fail(nullptr, MDAS_ERR_INVALID_ARG, "tune_batch: bad argument");
    for (int v = 0; v < n_waves; ++v)
        if (waves[v] < 0) return fail(nullptr, MDAS_ERR_INVALID_ARG, "tune_batch: a wave size is < 0");
    for (int v = 0; v < n_lanes; ++v)
        if (!nl_lanes_ok(lanes[v])) return fail(nullptr, MDAS_ERR_INVALID_ARG, "tune_batch: lanes must be 2 or 4");
    int best = -1;
    const int per_skin = 2 * n_waves * n_lanes;
    const int nc = n_skins * per_skin;
    for (int c = 0; c < nc; ++c) {
        const int ks = c / per_skin, kl = (c / (n_waves * n_lanes)) % 2, kw = (c / n_lanes) % n_waves,
                  kn = c % n_lanes;
        st = time_batch(descs, n_systems, skins[ks], kl, (long long)waves[kw], lanes[kn], md_steps, swap_trials,
                        rounds, &us_per_step[c]);
        if (st != MDAS_OK) return st;
        if (best < 0 || us_per_step[c] < us_per_step[best]) best = c;
    }
    *best_skin = skins[best / per_skin];
    *best_partitioned = (best / (n_waves * n_lanes)) % 2;
    *best_wave = waves[(best / n_lanes) % n_waves];
    *best_lanes = lanes[best % n_lanes];
    return MDAS_OK;
}

mdas_status mdas_set_batch_wave(mdas_system *s, int64_t max_beads) {
    if (!s || max_beads < 0) return fail(s, MDAS_ERR_INVALID_ARG, "set_batch_wave: bad argument");
    s->wave_beads = (long long)max_beads;
    return MDAS_OK;
}

mdas_status mdas_set_partitioned(mdas_system *s, int32_t enable) {
    if (!s) return fail(nullptr, MDAS_ERR_INVALID_ARG, "set_partitioned: NULL system");
    s->partition = enable != 0;
    return MDAS_OK;
}

mdas_status mdas_set_trial_path(mdas_system *s, int32_t path) {
    if (!s) return fail(nullptr, MDAS_ERR_INVALID_ARG, "set_trial_path: NULL system");
    if (path != MDAS_TRIALS_AUTO && path != MDAS_TRIALS_SPECULATIVE && path != MDAS_TRIALS_SEQUENTIAL)
        return fail(s, MDAS_ERR_INVALID_ARG, "set_trial_path: unknown path");
    s->trial_path = path;
    s->solo->trial_path = path;
    for (auto &kv : g_batches)
        if (kv.first[0] == s) kv.second->trial_path = path;
    return MDAS_OK;
}

mdas_status mdas_set_list_lanes(mdas_system *s, int32_t lanes) {
    if (!s) return fail(nullptr, MDAS_ERR_INVALID_ARG, "set_list_lanes: NULL system");
    if (!nl_lanes_ok(lanes)) return fail(s, MDAS_ERR_INVALID_ARG, "set_list_lanes: 2 or 4 list columns per bead");
    if (lanes == s->lanes) return MDAS_OK;
    const int before = s->lanes;
    s->lanes = lanes;
    // the system's own batch takes the new step shape (its step items change);
    // the pair list is built again at the next MD call
    mdas_status st = refill_batch(*s->solo, {s});
    if (st != MDAS_OK) s->lanes = before;
    return st;
}

mdas_status mdas_philox(uint32_t k0, uint32_t k1, uint32_t c1, uint32_t c2, uint32_t c3, int32_t n, uint32_t *out) {
    mdas_system *s = nullptr;
    if (n < 0 || (n > 0 && !out)) return fail(nullptr, MDAS_ERR_INVALID_ARG, "philox: bad argument");
    if (n == 0) return MDAS_OK;
    uint4 *d = nullptr;
    CK(cudaMalloc(&d, 16ull * n));
    launch_philox(k0, k1, c1, c2, c3, n, d, 0);
    cudaError_t e = cudaMemcpy(out, d, 16ull * n, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "philox");
    return MDAS_OK;
}

mdas_status mdas_set_kernel_timing(mdas_system *s, int32_t enable) {
    if (!s) return fail(nullptr, MDAS_ERR_INVALID_ARG, "set_kernel_timing: NULL system");
    s->timing = enable != 0;
    return MDAS_OK;
}

mdas_status mdas_set_soft_core(mdas_system *s, double delta) {
    if (!s || !(delta >= 0.0) || !std::isfinite(delta))
        return fail(s, MDAS_ERR_INVALID_ARG, "set_soft_core: delta must be finite and >= 0");
    s->hp.sc_delta = delta;
    s->hp.sc_deltaf = (float)delta;
    Params *dp = const_cast<Params *>(s->hs.p);
    CK(cudaMemcpyAsync(&dp->sc_delta, &s->hp.sc_delta, sizeof(double), cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(&dp->sc_deltaf, &s->hp.sc_deltaf, sizeof(float), cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return MDAS_OK;
}

mdas_status mdas_set_persistent(mdas_system *s, int32_t enable) {
    if (!s) return fail(nullptr, MDAS_ERR_INVALID_ARG, "set_persistent: NULL system");
    s->solo->persistent = enable != 0;
    return MDAS_OK;
}

mdas_status mdas_pair_kernel_time(mdas_system *s, double *total_ms, int64_t *launches, int32_t reset) {
    if (!s) return fail(nullptr, MDAS_ERR_INVALID_ARG, "pair_kernel_time: NULL system");
    if (total_ms) *total_ms = s->pair_ms;
    if (launches) *launches = s->pair_launches;
    if (reset) { s->pair_ms = 0.0; s->pair_launches = 0; }
    return MDAS_OK;
}

mdas_status mdas_get_counters(const mdas_system *cs, mdas_counters *out) {
    mdas_system *s = const_cast<mdas_system *>(cs);
    if (!s || !out) return fail(s, MDAS_ERR_INVALID_ARG, "get_counters: NULL argument");
    Counters c;
    CK(cudaMemcpyAsync(&c, s->hs.c, sizeof(c), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    out->md_steps = (int64_t)c.md_steps;
    out->force_evals = (int64_t)c.force_evals;
    out->trials = (int64_t)c.trials;
    out->null_trials = (int64_t)c.null_trials;
    out->accepted = (int64_t)c.accepted;
    out->moves = (int64_t)c.moves;
    out->moves_accepted = (int64_t)c.moves_accepted;
    out->kernel_launches = (int64_t)s->kernel_launches;
    out->list_builds = (int64_t)c.nl_builds;
    out->item_redos = (int64_t)c.redos;
    return MDAS_OK;
}

}  // extern "C"

// ================================================================= serving
// A request loop over device-resident systems (continuous batching): jobs are
// queued with a copy of their patch's description, admitted in arrival order
// while the device-memory budget and the slot count allow, and advanced in
// rounds in which one batched launch per phase covers every active job of a
// kind (MD jobs by a quantum of steps, swap jobs by their trials).  New jobs
// join at the next round; finished jobs leave and free their memory.  Every
// system keeps its own Philox key and counters, so a job's result does not
// depend on what else is running.

#include <chrono>
#include <deque>

namespace {

struct PendingJob {
    int64_t id = 0;
    int64_t patch = -1;                      // a resident patch, or -1: the job brings its own patch (d)
    mdas_job job{};
    double t_submit = 0.0;
    size_t footprint = 0;
    mdas_system_desc d{};
    std::vector<double> pos, vel, eps, sigma, charge;
    std::vector<int32_t> first, ltype, lbt, bonds, angles;
};

struct ActiveJob {
    PendingJob p;
    mdas_system *sys = nullptr;
    mdas_counters c0{};                      // the patch's counters when the job started (resident patches)
    double t_admit = 0.0;
    long long remaining = 0;
    bool done = false;
    double w = 0.0;
    int move_accepted = 0;
};

// arena bytes of a system (the sizes mdas_create_system allocates)
size_t arena_estimate(const mdas_system_desc *d) {
    const double shrink = grid_shrink(d);
    int nc = 1;
    for (int k = 0; k < 3; ++k) nc *= std::max(3, (int)std::floor(d->box[k] * (1.0 - shrink) / d->rc));
    const double mean = (double)d->n_beads / nc;
    const size_t capc = std::max(32, (int)std::ceil(4.0 * mean / 32.0) * 32);
    const size_t n = d->n_beads, vsz = d->precision == MDAS_FP64 ? 32 : 16;
    const size_t nbb = (n + BEAD_BLOCK - 1) / BEAD_BLOCK;
    size_t t = sizeof(Params) + sizeof(Counters) + 16 * n + vsz * n + 24 * n + 8 * std::max(d->n_lipids, 1) +
               8 * nc + 24 * nc * capc + vsz * nc * capc + 4 * n + 16 * nc + 24 * nbb + 32 * nc + 16 * n + vsz * n +
               (16 + 8 + 72 + 4 + 128 + 64) * (size_t)MAX_ROUND_TRIALS + sizeof(TrialRec) * (size_t)LOG_CAP + 512 +
               32 * MAX_DRAW_STEPS + 24 * n + 16 * std::max(d->n_lipids, 1) + 16 * RDF_MAX_BINS + 8;
    const ListDims ld = list_dims(d, shrink);
    t += 12ull * ld.n_lcells + 4ull * ld.n_lcells * ld.lcapc + 4 * n + 4 * n + 32 * n + 16 * n + 4ull * NL_LANES_MAX * n +
         4ull * ld.lcap * ld.npad + 4ull * NL_PART * n + 8ull * ((n + NL_BEADS_MIN - 1) / NL_BEADS_MIN / 32 + 1) +
         8ull * (n / NLB_BEADS + ld.n_lcells + 1);
    return t + 52 * 256;
}

}  // namespace

// A patch kept on the device between jobs: its state carries from one job
// to the next; one job at a time runs on it.
struct ResidentPatch {
    mdas_system *sys = nullptr;
    size_t footprint = 0;
    bool busy = false;                       // a job on it is active
    int queued = 0;                          // jobs on it waiting in the queue
};

struct mdas_server {
    std::map<int64_t, ResidentPatch> patches;
    int64_t next_patch = 1;
    size_t budget = 0, in_use = 0;
    int max_active = 0;
    int md_quantum = 25;
    int want_state = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t upload = nullptr;           // uploads of admitted patches, beside the round's device work
    std::deque<PendingJob> queue;
    std::vector<ActiveJob> active;
    std::vector<mdas_job_result> finished;
    Batch md_batch, swap_batch, mdas_batch, mdas_run_batch;
    int64_t next_id = 1;
    std::chrono::steady_clock::time_point t0;
    std::multimap<size_t, void *> pool;      // freed arenas by size, reused by later jobs
    std::map<void *, size_t> sizes;
    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

void *pool_alloc(size_t bytes, void *, void *ctx) {
    mdas_server *sv = (mdas_server *)ctx;
    auto it = sv->pool.lower_bound(bytes);
    if (it != sv->pool.end() && it->first <= 2 * bytes) {
        void *p = it->second;
        sv->pool.erase(it);
        return p;
    }
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    sv->sizes[p] = bytes;
    return p;
}

void pool_free(void *p, void *, void *ctx) {
    mdas_server *sv = (mdas_server *)ctx;
    sv->pool.emplace(sv->sizes[p], p);
}

uint64_t fnv1a(uint64_t h, const void *data, size_t n) {
    const unsigned char *c = (const unsigned char *)data;
    for (size_t k = 0; k < n; ++k) { h ^= c[k]; h *= 1099511628211ull; }
    return h;
}

mdas_status finish_job(mdas_server *sv, ActiveJob &a) {
    mdas_system *s = a.sys;
    const bool resident = a.p.patch >= 0;
    mdas_job_result r{};
    r.job_id = a.p.id;
    r.kind = a.p.job.kind;
    r.status = MDAS_OK;
    r.t_submit = a.p.t_submit;
    r.t_admit = a.t_admit;
    mdas_counters c{};
    mdas_status st = mdas_get_counters(s, &c);
    if (st != MDAS_OK) return st;
    r.t_done = sv->now();
    r.md_steps = c.md_steps - a.c0.md_steps;
    r.trials = c.trials - a.c0.trials;
    r.accepted = c.accepted - a.c0.accepted;
    r.w = a.w;
    r.move_accepted = a.move_accepted;
    if (sv->want_state) {
        std::vector<uint32_t> pu(3ull * s->n);
        std::vector<double> v(3ull * s->n);
        std::vector<int32_t> lt(std::max(s->n_lip, 1));
        mdas_state_view sv_{};
        sv_.pos_fixed = pu.data();
        sv_.vel = v.data();
        sv_.lipid_type = lt.data();
        st = mdas_get_state(s, &sv_);
        if (st != MDAS_OK) return st;
        uint64_t h = 1469598103934665603ull;
        h = fnv1a(h, pu.data(), 4ull * pu.size());
        h = fnv1a(h, v.data(), 8ull * v.size());
        h = fnv1a(h, lt.data(), 4ull * s->n_lip);
        r.state_hash = h;
    }
    if (resident) {
        sv->patches[a.p.patch].busy = false;
    } else {
        sv->in_use -= a.p.footprint;
        mdas_destroy_system(s);
    }
    a.sys = nullptr;
    sv->finished.push_back(r);
    return MDAS_OK;
}

// A system created from a copy of a description for the server: uploads on
// the upload stream, then working on the server's stream.
mdas_status server_create(mdas_server *sv, const PendingJob &p, mdas_system **out) {
    mdas_system_desc d = p.d;
    d.pos = p.pos.data();
    d.vel = p.vel.empty() ? nullptr : p.vel.data();
    d.eps = p.eps.data(); d.sigma = p.sigma.data(); d.charge = p.charge.data();
    d.lipid_first_bead = p.first.empty() ? nullptr : p.first.data();
    d.lipid_type = p.ltype.data();
    d.lipid_bead_type = p.lbt.data();
    d.bonds = p.bonds.empty() ? nullptr : p.bonds.data();
    d.angles = p.angles.empty() ? nullptr : p.angles.data();
    d.cuda_stream = sv->upload;
    d.dev_alloc = pool_alloc;
    d.dev_free = pool_free;
    d.alloc_ctx = sv;
    mdas_status st = mdas_create_system(&d, out);
    if (st != MDAS_OK) return st;
    // creation waited for its uploads: from here on the server's stream
    (*out)->stream = sv->stream;
    (*out)->solo->stream = sv->stream;
    return MDAS_OK;
}

// A host copy of a description's arrays (the job or patch keeps them).
mdas_status copy_desc(const mdas_system_desc *d, PendingJob &p) {
    if (!d || d->n_beads <= 0 || !d->pos || !d->lipid_type || !d->lipid_bead_type || !d->eps || !d->sigma || !d->charge)
        return MDAS_ERR_INVALID_ARG;
    const size_t n = d->n_beads, nl = d->n_lipids, nbt = d->n_bead_types;
    p.pos.assign(d->pos, d->pos + 3 * n);
    if (d->vel) p.vel.assign(d->vel, d->vel + 3 * n);
    p.eps.assign(d->eps, d->eps + nbt * nbt);
    p.sigma.assign(d->sigma, d->sigma + nbt * nbt);
    p.charge.assign(d->charge, d->charge + nbt);
    if (d->lipid_first_bead) p.first.assign(d->lipid_first_bead, d->lipid_first_bead + nl);
    p.ltype.assign(d->lipid_type, d->lipid_type + nl);
    p.lbt.assign(d->lipid_bead_type, d->lipid_bead_type + (size_t)d->n_lipid_types * d->beads_per_lipid);
    if (d->n_bonds) p.bonds.assign(d->bonds, d->bonds + 2 * d->n_bonds);
    if (d->n_angles) p.angles.assign(d->angles, d->angles + 3 * d->n_angles);
    p.d = *d;
    return MDAS_OK;
}

// Admit queued jobs in arrival order while a slot and room in the memory
// budget are free.  A patch is created with its uploads on the upload stream,
// so they run beside whatever the round has already launched on the server's
// stream; the system then works on the server's stream.
mdas_status admit(mdas_server *sv, bool resident_only) {
    for (auto it = sv->queue.begin(); it != sv->queue.end() && (int)sv->active.size() < sv->max_active;) {
        PendingJob &q = *it;
        ActiveJob a;
        if (q.patch < 0 && resident_only) { ++it; continue; }
        if (q.patch >= 0) {
            // a job on a resident patch: its patch must be idle (jobs on one
            // patch run one after another, in submission order)
            ResidentPatch &rp = sv->patches[q.patch];
            if (rp.busy) { ++it; continue; }
            rp.busy = true;
            rp.queued--;
            a.sys = rp.sys;
            mdas_status st = mdas_get_counters(a.sys, &a.c0);
            if (st != MDAS_OK) return st;
        } else {
            // a job with its own patch: created now if the memory budget allows
            // (arrival order: a job that does not fit waits, and so do the jobs
            // with their own patches behind it)
            if (sv->in_use + q.footprint > sv->budget) break;
            mdas_status st = server_create(sv, q, &a.sys);
            if (st != MDAS_OK) return st;
            sv->in_use += q.footprint;
        }
        a.t_admit = sv->now();
        a.remaining = q.job.kind == MDAS_JOB_MD ? q.job.n : 1;
        a.p = std::move(q);
        it = sv->queue.erase(it);
        sv->active.push_back(std::move(a));
    }
    return MDAS_OK;
}

// The MDAS jobs of one parameter set (pairs, lambda steps, MD steps per
// lambda) as one batched move: every launch of mdas_alchemical_move covers
// all of them (pair selection, the alchemical trajectory of those that found
// pairs in one MD run, the Metropolis test, the restore).  Per system the
// arithmetic is that of its own move.
mdas_status batched_moves(mdas_server *sv, const std::vector<ActiveJob *> &jobs) {
    const mdas_job &j = jobs[0]->p.job;
    std::vector<mdas_system *> v;
    for (auto *a : jobs) v.push_back(a->sys);
    mdas_system *s = v[0];                    // where errors are reported
    mdas_status st = refill_batch(sv->mdas_batch, v);
    if (st != MDAS_OK) return st;
    LaunchCtx L = sv->mdas_batch.ctx();
    launch_snapshot(L);
    launch_mdas_select(L, j.n_pairs, 64 * j.n_pairs + 64, 0);
    std::vector<int> np(v.size(), 0);
    for (size_t k = 0; k < v.size(); ++k)
        CK(cudaMemcpyAsync(&np[k], &v[k]->hs.c->n_pairs, 4, cudaMemcpyDeviceToHost, sv->stream));
    CK(cudaStreamSynchronize(sv->stream));
    std::vector<mdas_system *> run;
    for (size_t k = 0; k < v.size(); ++k)
        if (np[k] > 0) run.push_back(v[k]);
    if (!run.empty()) {
        st = refill_batch(sv->mdas_run_batch, run);
        if (st != MDAS_OK) return st;
        LaunchCtx R = sv->mdas_run_batch.ctx();
        const double dl = 1.0 / j.n_lambda;
        if (j.md_per_lambda > 0) {
            launch_mdas_set_lambda(R, 0.0, 1);
            st = run_md(run[0], sv->mdas_run_batch, (long long)j.n_lambda * j.md_per_lambda, 0, true, false,
                        j.md_per_lambda, dl);
            if (st != MDAS_OK) return st;
        } else {
            for (int k = 1; k <= j.n_lambda; ++k) {
                launch_mdas_set_lambda(R, (double)(k - 1) / j.n_lambda, 1);
                st = build_cells(run[0], sv->mdas_run_batch);
                if (st != MDAS_OK) return st;
                launch_mdas_dE(R, dl);
            }
        }
    }
    launch_mdas_accept(L);
    launch_mdas_restore(L);
    std::vector<Counters> c(v.size());
    for (size_t k = 0; k < v.size(); ++k)
        CK(cudaMemcpyAsync(&c[k], v[k]->hs.c, sizeof(Counters), cudaMemcpyDeviceToHost, sv->stream));
    CK(cudaStreamSynchronize(sv->stream));
    CK(cudaGetLastError());
    for (size_t k = 0; k < v.size(); ++k) {
        v[k]->cells_valid = false;
        jobs[k]->w = c[k].w;
        jobs[k]->move_accepted = c[k].mdas_accept;
    }
    return check_err(v[0], sv->mdas_batch);
}

}  // namespace

extern "C" {

mdas_status mdas_server_create(size_t hbm_budget_bytes, int32_t max_active, int32_t md_quantum, int32_t keep_state_hash,
                               void *cuda_stream, mdas_server **out) {
    if (!out || hbm_budget_bytes == 0 || max_active <= 0 || md_quantum <= 0)
        return fail(nullptr, MDAS_ERR_INVALID_ARG, "server_create: bad argument");
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    if (!stream) {
        cudaError_t e = shared_stream(&stream);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "server_create: stream");
    }
    mdas_server *sv = new mdas_server();
    sv->budget = hbm_budget_bytes;
    sv->max_active = max_active;
    sv->md_quantum = md_quantum;
    sv->want_state = keep_state_hash;
    sv->stream = stream;
    {
        cudaError_t e = cudaStreamCreateWithFlags(&sv->upload, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete sv;
            return cuda_fail(nullptr, e, "server_create: upload stream");
        }
    }
    sv->t0 = std::chrono::steady_clock::now();
    *out = sv;
    return MDAS_OK;
}

void mdas_server_destroy(mdas_server *sv) {
    if (!sv) return;
    for (auto &a : sv->active)
        if (a.sys && a.p.patch < 0) mdas_destroy_system(a.sys);
    for (auto &kv : sv->patches) mdas_destroy_system(kv.second.sys);
    cudaStreamSynchronize(sv->stream);
    for (auto &kv : sv->sizes) cudaFree(kv.first);
    destroy_batch(&sv->md_batch);
    destroy_batch(&sv->swap_batch);
    destroy_batch(&sv->mdas_batch);
    destroy_batch(&sv->mdas_run_batch);
    if (sv->upload) cudaStreamDestroy(sv->upload);
    delete sv;
}

namespace {

bool job_ok(const mdas_job *job) {
    return job && job->kind >= MDAS_JOB_SWAPS && job->kind <= MDAS_JOB_MDAS && job->n >= 0 &&
           !(job->kind == MDAS_JOB_MDAS &&
             (job->n_pairs < 0 || job->n_pairs > MAX_PAIRS || job->n_lambda < 1 || job->md_per_lambda < 0));
}

}  // namespace

mdas_status mdas_server_submit(mdas_server *sv, const mdas_system_desc *d, const mdas_job *job, int64_t *job_id) {
    if (!sv || !d || !job) return fail(nullptr, MDAS_ERR_INVALID_ARG, "server_submit: bad argument");
    if (!job_ok(job)) return fail(nullptr, MDAS_ERR_INVALID_ARG, "server_submit: bad job");
    PendingJob p;
    if (copy_desc(d, p) != MDAS_OK) return fail(nullptr, MDAS_ERR_INVALID_ARG, "server_submit: bad argument");
    p.footprint = arena_estimate(d);
    if (p.footprint > sv->budget) return fail(nullptr, MDAS_ERR_OOM, "server_submit: the job alone exceeds the memory budget");
    p.id = sv->next_id++;
    p.job = *job;
    p.t_submit = sv->now();
    if (job_id) *job_id = p.id;
    sv->queue.push_back(std::move(p));
    return MDAS_OK;
}

mdas_status mdas_server_add_patch(mdas_server *sv, const mdas_system_desc *d, int64_t *patch_id) {
    if (!sv || !d || !patch_id) return fail(nullptr, MDAS_ERR_INVALID_ARG, "server_add_patch: bad argument");
    PendingJob p;
    if (copy_desc(d, p) != MDAS_OK) return fail(nullptr, MDAS_ERR_INVALID_ARG, "server_add_patch: bad argument");
    const size_t fp = arena_estimate(d);
    if (sv->in_use + fp > sv->budget)
        return fail(nullptr, MDAS_ERR_OOM, "server_add_patch: the patch does not fit the free memory budget");
    ResidentPatch rp;
    mdas_status st = server_create(sv, p, &rp.sys);
    if (st != MDAS_OK) return st;
    rp.footprint = fp;
    sv->in_use += fp;
    *patch_id = sv->next_patch++;
    sv->patches[*patch_id] = rp;
    return MDAS_OK;
}

mdas_status mdas_server_submit_to(mdas_server *sv, int64_t patch_id, const mdas_job *job, int64_t *job_id) {
    if (!sv || !job) return fail(nullptr, MDAS_ERR_INVALID_ARG, "server_submit_to: bad argument");
    if (!job_ok(job)) return fail(nullptr, MDAS_ERR_INVALID_ARG, "server_submit_to: bad job");
    auto it = sv->patches.find(patch_id);
    if (it == sv->patches.end()) return fail(nullptr, MDAS_ERR_INVALID_ARG, "server_submit_to: no such patch");
    PendingJob p;
    p.id = sv->next_id++;
    p.patch = patch_id;
    p.job = *job;
    p.t_submit = sv->now();
    it->second.queued++;
    if (job_id) *job_id = p.id;
    sv->queue.push_back(std::move(p));
    return MDAS_OK;
}

mdas_status mdas_server_remove_patch(mdas_server *sv, int64_t patch_id) {
    if (!sv) return fail(nullptr, MDAS_ERR_INVALID_ARG, "server_remove_patch: bad argument");
    auto it = sv->patches.find(patch_id);
    if (it == sv->patches.end()) return fail(nullptr, MDAS_ERR_INVALID_ARG, "server_remove_patch: no such patch");
    if (it->second.busy || it->second.queued > 0)
        return fail(nullptr, MDAS_ERR_BUSY, "server_remove_patch: the patch has active or queued jobs");
    sv->in_use -= it->second.footprint;
    mdas_destroy_system(it->second.sys);
    sv->patches.erase(it);
    return MDAS_OK;
}

mdas_status mdas_server_patch_state(mdas_server *sv, int64_t patch_id, mdas_state_view *out) {
    if (!sv || !out) return fail(nullptr, MDAS_ERR_INVALID_ARG, "server_patch_state: bad argument");
    auto it = sv->patches.find(patch_id);
    if (it == sv->patches.end()) return fail(nullptr, MDAS_ERR_INVALID_ARG, "server_patch_state: no such patch");
    if (it->second.busy) return fail(nullptr, MDAS_ERR_BUSY, "server_patch_state: a job is running on the patch");
    return mdas_get_state(it->second.sys, out);
}

mdas_status mdas_server_run(mdas_server *sv, int32_t max_rounds, int32_t *n_active, int32_t *n_queued) {
    if (!sv || max_rounds < 0) return fail(nullptr, MDAS_ERR_INVALID_ARG, "server_run: bad argument");
    for (int r = 0; r < max_rounds; ++r) {
        // jobs on resident patches join at once (nothing to create); an idle
        // server admits every kind at once (there is no work to overlap with)
        {
            mdas_status st = admit(sv, !sv->active.empty());
            if (st != MDAS_OK) return st;
        }
        if (sv->active.empty()) break;
        // MD jobs: one batched quantum of steps, launched without waiting
        std::vector<mdas_system *> mdv;
        long long q = sv->md_quantum;
        for (auto &a : sv->active)
            if (a.p.job.kind == MDAS_JOB_MD && a.remaining > 0) { mdv.push_back(a.sys); q = std::min(q, a.remaining); }
        if (!mdv.empty()) {
            mdas_status st = refill_batch(sv->md_batch, mdv);
            if (st == MDAS_OK) st = run_md(mdv[0], sv->md_batch, q, 0, false, false);
            if (st != MDAS_OK) return st;
            for (auto &a : sv->active)
                if (a.p.job.kind == MDAS_JOB_MD && a.remaining > 0) {
                    a.remaining -= q;
                    if (a.remaining == 0) a.done = true;
                }
        }
        // jobs that arrived meanwhile, created while the quantum runs; new MD
        // jobs start with the next round, new swap and MDAS jobs below
        {
            mdas_status st = admit(sv, false);
            if (st != MDAS_OK) return st;
        }
        // swap jobs: one batched evaluation per trial count
        std::map<int, std::vector<ActiveJob *>> groups;
        for (auto &a : sv->active)
            if (a.p.job.kind == MDAS_JOB_SWAPS && !a.done) groups[a.p.job.n].push_back(&a);
        for (auto &g : groups) {
            std::vector<mdas_system *> v;
            for (auto *a : g.second)
                if (a->sys->n_lip > 0) v.push_back(a->sys);
            if (!v.empty() && g.first > 0) {
                mdas_status st = refill_batch(sv->swap_batch, v);
                if (st == MDAS_OK) st = run_trials(v[0], sv->swap_batch, g.first, nullptr);
                if (st != MDAS_OK) return st;
            }
            for (auto *a : g.second) a->done = true;
        }
        // MDAS jobs: one batched move per parameter set
        std::map<std::vector<int>, std::vector<ActiveJob *>> moves;
        for (auto &a : sv->active)
            if (a.p.job.kind == MDAS_JOB_MDAS && !a.done) {
                a.done = true;
                if (a.sys->n_lip > 0)
                    moves[{a.p.job.n_pairs, a.p.job.n_lambda, a.p.job.md_per_lambda}].push_back(&a);
            }
        for (auto &g : moves) {
            mdas_status st = batched_moves(sv, g.second);
            if (st != MDAS_OK) return st;
        }
        // completion: errors of the MD quantum, results, memory back to the pool, slots free
        if (!mdv.empty()) {
            mdas_status st = check_err(mdv[0], sv->md_batch);
            if (st != MDAS_OK) return st;
        }
        {
            cudaError_t e = cudaStreamSynchronize(sv->stream);
            if (e != cudaSuccess) return cuda_fail(nullptr, e, "server_run");
        }
        std::vector<ActiveJob> keep;
        for (auto &a : sv->active) {
            if (a.done) {
                mdas_status st = finish_job(sv, a);
                if (st != MDAS_OK) return st;
            } else {
                keep.push_back(std::move(a));
            }
        }
        sv->active.swap(keep);
    }
    if (n_active) *n_active = (int32_t)sv->active.size();
    if (n_queued) *n_queued = (int32_t)sv->queue.size();
    return MDAS_OK;
}

mdas_status mdas_server_results(mdas_server *sv, mdas_job_result *out, int32_t cap, int32_t *n) {
    if (!sv || !n || cap < 0 || (cap > 0 && !out)) return fail(nullptr, MDAS_ERR_INVALID_ARG, "server_results: bad argument");
    const int m = std::min<int>(cap, (int)sv->finished.size());
    for (int k = 0; k < m; ++k) out[k] = sv->finished[k];
    sv->finished.erase(sv->finished.begin(), sv->finished.begin() + m);
    *n = m;
    return MDAS_OK;
}

double mdas_server_clock(const mdas_server *sv) { return sv ? sv->now() : 0.0; }

size_t mdas_system_footprint(const mdas_system_desc *d) {
    if (!d || d->n_beads <= 0 || !(d->rc > 0)) return 0;
    return arena_estimate(d);
}

}  // extern "C"
