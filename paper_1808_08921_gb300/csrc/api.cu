// api.cu -- the C ABI (include/lbmdem.h): context, layout orchestration, the
// coupled step loop (CUDA graphs of several steps), re-layouts and read-outs.
//
// One coupled step t -> t+1 on the context stream (Sections 2.1-2.4):
//   map update (re-test band nodes, convert covered/uncovered nodes)
//   collide + stream (even or odd AA kernel)
//   link bounce-back + hydrodynamic force and torque
//   inlet / outlet
//   K DEM substeps (one cluster launch; also advances the device step counter)
// Steps are captured in CUDA graphs of `graph_steps` steps starting at even t.
// With mobile spheres the host reads back the largest displacement since the
// last re-layout every few graphs and rebuilds the compact lattice and the
// neighbour lists before any sphere can leave its skin.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <cuda.h>
#include <string>
#include <vector>

#include "../../include/lbmdem.h"
#include "common.cuh"
#include "kernels.cuh"
#include "layout.cuh"

using namespace lbmdem;

namespace {

template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    ~DBuf() { release(); }
    cudaError_t alloc(size_t count) {
        release();
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc((void**)&p, sizeof(T) * count);
        if (e != cudaSuccess) {
            p = nullptr;
            n = 0;
            return e;
        }
        n = count;
        return cudaSuccess;
    }
    cudaError_t ensure(size_t count) { return count <= n && p ? cudaSuccess : alloc(count + count / 8); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void swap(DBuf& o) {
        std::swap(p, o.p);
        std::swap(n, o.n);
    }
};

constexpr int NGROUP = 6;  // collide odd, links, map update, inlet/outlet, DEM, collide even

}  // namespace

// cell-list buffers (per-sphere cell, per-cell counts, starts, fill cursors
// and the spheres in cell order)
struct CellBufs {
    DBuf<int> of, count, start, fill, order;
};

struct lbmdem_ctx {
    lbmdem_params p{};
    std::string err;
    int status_latched = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t side = nullptr;             // inlet/outlet, beside the DEM
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int nw = 0;
    size_t N = 0, W = 0;
    bool lbm = true;
    bool have_packing = false;
    int64_t t = 0;
    Source src{};
    double skin = 0.25, dem_skin = 0.5, trigger = 0.0, hard = 0.0;
    // lattice
    DBuf<int32_t> owner;
    DBuf<unsigned long long> paint_best;
    DBuf<uint8_t> deep, band;
    DBuf<uint4> rec, rec2;
    DBuf<uint32_t> maskB, maskB2, cntA, cntB, scan_tmp;
    DBuf<uint8_t> f, f2;  // populations, 4 or 2 bytes each
    DBuf<uint32_t> coord, fbits;
    uint32_t nA = 0, nS = 0, nSpad = 0;
    DBuf<uint32_t> band_coord, band_count, band_coord2, slack_hist;
    DBuf<int4> band_cand, band_cand2;
    DBuf<float> band_slack, band_slack2;
    uint32_t nband = 0;
    DBuf<uint32_t> surf_count, surf_off;
    DBuf<uint2> surf_link;
    DBuf<uint32_t> warp_p;
    DBuf<uint8_t> chunk_dir;  // direction (| flag) of every 32-record chunk
    uint32_t nwarps = 0;
    uint32_t nlink_raw = 0;  // link records before padding
    DBuf<uint2> linkw;       // link word of every stored node (even steps' links in the collide kernel)
    bool fused_links = false;
    bool batched = false;  // steps being captured into a batch graph (columns share the GPU)
    DBuf<Flip> flip_rec;
    DBuf<float> flip_scratch;
    DBuf<uint8_t> flip_valid;
    uint32_t flip_cap = 0;
    uint32_t pA0 = 0, pA1 = 0, pB0 = 0, pB1 = 0;
    // particles
    int np = 0;
    bool any_mobile = false;
    double Rmax = 0;
    DBuf<double> Xref, Fh, Th, Rd, Fh_prev, Th_prev;
    DBuf<float4> Fa, Ta;
    DBuf<float4> dX, dXc, dXb, V, Om, q, Vhb, Whb, Fc, Tc, xf;
    DBuf<float4> ab;  // [n][Q-1] per-step link terms, written by the map update
    DBuf<float4> pk;  // [n][3] per-step sphere packets, written by the map update
    DBuf<int4> org, orgw;
    DBuf<float> R, invm, invI;
    DBuf<uint8_t> fixed;
    int nbmax = 48;
    DBuf<int> nb_cnt, nb_j, nb_cnt2, nb_j2;
    DBuf<int8_t> nb_sh, nb_sh2;
    DBuf<float4> nb_dref, nb_ft, nb_dref2, nb_ft2;
    CellGrid grid{};
    CellBufs cells;       // the DEM's cell list (cells 2 R + dem_skin wide)
    CellBufs band_cells;  // cells R + skin wide: a band node's candidates lie within R + skin
    // stats, probe
    DBuf<DevStats> st;
    DevStats* st_host = nullptr;
    DBuf<double> probe;
    size_t probe_cap = 0;
    int64_t mon_step = -1;
    // timing
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_group;  // group of each recorded pair (pairs = ev[2k], ev[2k+1])
    size_t ev_pairs = 0;
    size_t gpairs = 0;                  // event pairs recorded by one graph launch
    std::vector<int> gev_group;
    double tm_ms[NGROUP] = {0};
    int64_t tm_n[NGROUP] = {0};
    // graph
    cudaGraphExec_t gexec = nullptr;
    int glen = 16;
    bool gtiming = false;
    int64_t relayouts = 0;
    int64_t steps_until_check = 0;
    bool capturing = false;      // inside stream capture (events become graph nodes)
    bool suppress_probe = false; // re-running steps whose probe trace is recorded
    int64_t launches = 0;        // kernels enqueued by the step loop
    int64_t glaunches = 0;       // kernels in one captured graph
};

// ------------------------------------------------------------ helpers

static int fail(lbmdem_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(c, e_ == cudaErrorMemoryAllocation ? LBMDEM_ERR_OOM : LBMDEM_ERR_CUDA,     \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);      \
    } while (0)

static int map_status(uint32_t s) {
    if (s & ST_UNSTABLE) return LBMDEM_ERR_UNSTABLE;
    if (s & ST_SKIN) return LBMDEM_ERR_SKIN;
    if (s & ST_CAPACITY) return LBMDEM_ERR_CAPACITY;
    if (s & ST_TIMEOUT) return LBMDEM_ERR_TIMEOUT;
    return 0;
}

static const char* status_text(int code) {
    switch (code) {
        case LBMDEM_ERR_UNSTABLE: return "device status: NaN/Inf in the fluid or the spheres";
        case LBMDEM_ERR_SKIN: return "device status: a sphere moved beyond the re-layout skin";
        case LBMDEM_ERR_CAPACITY: return "device status: a device list overflowed";
        case LBMDEM_ERR_TIMEOUT: return "device status: a bounded wait gave up";
    }
    return "";
}

static Lat make_lat(lbmdem_ctx* c) {
    Lat L{};
    L.nx = c->p.nx;
    L.ny = c->p.ny;
    L.nz = c->p.nz;
    L.nw = c->nw;
    L.px = c->p.inlet == LBMDEM_X_PERIODIC;
    L.nA = c->nA;
    L.nS = c->nS;
    L.nSpad = c->nSpad;
    L.f = c->f.p;
    L.st = c->p.storage == LBMDEM_BF16_DEV ? 1 : c->p.storage == LBMDEM_F16_DEV ? 2 : 0;
    L.fs = L.st == 2 ? 4096.0f : 1.0f;  // FP16: deviations 1e-8 .. 16 stay normal
    L.fsi = 1.0f / L.fs;
    L.rec = c->rec.p;
    L.maskB = c->maskB.p;
    L.coord = c->coord.p;
    L.fbits = c->fbits.p;
    L.owner = c->owner.p;
    L.tau_inv = (float)(1.0 / c->p.tau);
    L.rho_f = (float)c->p.rho_f;
    return L;
}

static PartView make_part(lbmdem_ctx* c) {
    PartView P{};
    P.n = c->np;
    P.Xref = c->Xref.p;
    P.dX = c->dX.p;
    P.dXc = c->dXc.p;
    P.V = c->V.p;
    P.W = c->Om.p;
    P.R = c->R.p;
    P.Rd = c->Rd.p;
    P.org = c->org.p;
    P.orgw = c->orgw.p;
    P.xf = c->xf.p;
    P.ab = c->ab.p;
    P.pk = c->pk.p;
    P.Fh = c->Fh.p;
    P.Th = c->Th.p;
    return P;
}

static Dem make_dem(lbmdem_ctx* c) {
    Dem D{};
    D.n = c->np;
    D.K = c->p.dem_substeps;
    D.cluster = 8;
    D.dt = 1.0f / (float)c->p.dem_substeps;
    D.kn = (float)(2.0 * c->p.E_p / (3.0 * (1.0 - c->p.nu_p * c->p.nu_p)));
    D.kt = (float)(2.0 * c->p.E_p / ((1.0 + c->p.nu_p) * (2.0 - c->p.nu_p)));
    D.mu = (float)c->p.mu;
    D.g = make_float3((float)c->p.body_force[0], (float)c->p.body_force[1], (float)c->p.body_force[2]);
    D.nbmax = c->nbmax;
    D.Xref = c->Xref.p;
    D.dX = c->dX.p;
    D.dXc = c->dXc.p;
    D.dXb = c->dXb.p;
    D.V = c->V.p;
    D.W = c->Om.p;
    D.q = c->q.p;
    D.Vhb = c->Vhb.p;
    D.Whb = c->Whb.p;
    D.Fc = c->Fc.p;
    D.Tc = c->Tc.p;
    D.Fh = c->Fh.p;
    D.Th = c->Th.p;
    D.Fh_prev = c->Fh_prev.p;
    D.Th_prev = c->Th_prev.p;
    D.Fa = c->Fa.p;
    D.Ta = c->Ta.p;
    D.R = c->R.p;
    D.invm = c->invm.p;
    D.invI = c->invI.p;
    D.fixed = c->fixed.p;
    D.nb_cnt = c->nb_cnt.p;
    D.nb_j = c->nb_j.p;
    D.nb_dref = c->nb_dref.p;
    D.nb_ft = c->nb_ft.p;
    D.org = c->org.p;
    D.orgw = c->orgw.p;
    D.xf = c->xf.p;
    DevStats* s = c->st.p;
    D.status = &s->status;
    D.max_disp_bits = &s->max_disp_bits;
    D.disp_layout_bits = &s->disp_layout_bits;
    D.layout_fresh = &s->layout_fresh;
    D.max_vel_bits = &s->max_vel_bits;
    D.hard_disp = (float)c->hard;
    D.px = c->p.inlet == LBMDEM_X_PERIODIC;
    D.Lx = c->p.nx;
    D.Ly = c->p.ny;
    D.Lz = c->p.nz;
    return D;
}

static void destroy_graph(lbmdem_ctx* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
}

// ------------------------------------------------------------ layout build

// A cell list of the reference centres with cells at least h wide.
static int build_cell_grid(lbmdem_ctx* c, CellGrid& G, double h, CellBufs& B) {
    int np = c->np;
    if (h <= 0) h = 1.0;
    int px = c->p.inlet == LBMDEM_X_PERIODIC;
    G.px = px;
    G.L = make_double3(c->p.nx, c->p.ny, c->p.nz);
    if (px) {
        G.nc.x = std::max(1, (int)floor(c->p.nx / h));
        G.lo.x = 0;
        G.h.x = (double)c->p.nx / G.nc.x;
    } else {
        double lo = -(c->Rmax + 2.0), hi = c->p.nx + c->Rmax + 2.0;
        G.nc.x = std::max(1, (int)floor((hi - lo) / h));
        G.lo.x = lo;
        G.h.x = (hi - lo) / G.nc.x;
    }
    G.nc.y = std::max(1, (int)floor(c->p.ny / h));
    G.h.y = (double)c->p.ny / G.nc.y;
    G.nc.z = std::max(1, (int)floor(c->p.nz / h));
    G.h.z = (double)c->p.nz / G.nc.z;
    G.lo.y = G.lo.z = 0;
    int ncell = G.nc.x * G.nc.y * G.nc.z;
    CK(B.of.ensure(np));
    CK(B.count.ensure(ncell + 1));
    CK(c->scan_tmp.ensure(scan_tmp_size((size_t)ncell + 1)));  // allocated at init with a lattice
    CK(B.start.ensure(ncell + 1));
    CK(B.fill.ensure(ncell));
    CK(B.order.ensure(np));
    launch_cells(c->Xref.p, np, G, B.of.p, B.count.p, B.start.p, B.fill.p, B.order.p, c->scan_tmp.p, c->stream);
    CK(cudaGetLastError());
    return 0;
}

// the DEM's cells: a contact partner lies within 2 R + dem_skin
static int build_cells(lbmdem_ctx* c) { return build_cell_grid(c, c->grid, 2.0 * c->Rmax + c->dem_skin, c->cells); }

// neighbour lists from Xref; `carry` keeps the tangential history
static int build_neighbours(lbmdem_ctx* c, bool carry) {
    int np = c->np;
    size_t ne = (size_t)std::max(np, 1) * c->nbmax;
    CK(c->nb_cnt2.ensure(np));
    CK(c->nb_j2.ensure(ne));
    CK(c->nb_sh2.ensure(4 * ne));
    CK(c->nb_dref2.ensure(ne));
    CK(c->nb_ft2.ensure(ne));
    NbBuild B{};
    B.X = c->Xref.p;
    B.R = c->Rd.p;
    B.n = np;
    B.nbmax = c->nbmax;
    B.skin = c->dem_skin;
    B.G = c->grid;
    B.start = c->cells.start.p;
    B.order = c->cells.order.p;
    B.cnt = c->nb_cnt2.p;
    B.nj = c->nb_j2.p;
    B.nsh = c->nb_sh2.p;
    B.dref = c->nb_dref2.p;
    B.ft = c->nb_ft2.p;
    bool have_old = carry && c->nb_cnt.p && c->nb_cnt.n >= (size_t)np;
    B.old_cnt = have_old ? c->nb_cnt.p : nullptr;
    B.old_j = have_old ? c->nb_j.p : nullptr;
    B.old_sh = have_old ? c->nb_sh.p : nullptr;
    B.old_ft = have_old ? c->nb_ft.p : nullptr;
    B.status = &c->st.p->status;
    launch_nb_build(B, c->stream);
    CK(cudaGetLastError());
    c->nb_cnt.swap(c->nb_cnt2);
    c->nb_j.swap(c->nb_j2);
    c->nb_sh.swap(c->nb_sh2);
    c->nb_dref.swap(c->nb_dref2);
    c->nb_ft.swap(c->nb_ft2);
    return 0;
}

static int read_u32(lbmdem_ctx* c, const uint32_t* d, uint32_t* h) {
    CK(cudaMemcpyAsync(h, d, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return 0;
}

// Compact lattice from Xref.  fresh: fluid at rest; else copy the populations
// from the current layout (the state must be between an odd and an even step).
static int build_layout(lbmdem_ctx* c, bool fresh) {
    cudaStream_t s = c->stream;
    int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    int px = c->p.inlet == LBMDEM_X_PERIODIC;
    if (fresh) fill_i32(c->owner.p, OWNER_FLUID, c->N, s);
    CK(cudaMemsetAsync(c->deep.p, 0, c->N, s));
    CK(cudaMemsetAsync(c->band.p, 0, c->N, s));
    if (fresh) CK(c->paint_best.alloc(c->N));
    PaintArgs PA{c->Xref.p, c->Rd.p, nx, ny, nz, px, c->skin, fresh ? c->owner.p : nullptr,
                 fresh ? c->paint_best.p : nullptr, c->deep.p, c->band.p};
    launch_paint(PA, c->np, c->N, s);
    CK(cudaGetLastError());
    if (fresh) {
        CK(cudaStreamSynchronize(s));
        c->paint_best.release();
    }
    // words into the spare record set (the current one is needed for the copy)
    LayoutArgs LA{nx, ny, nz, c->nw, c->owner.p, c->deep.p, c->band.p, c->rec2.p, c->maskB2.p,
                  c->cntA.p, c->cntB.p, nullptr};
    CK(cudaMemsetAsync(c->cntA.p, 0, sizeof(uint32_t) * (c->W + 1), s));
    CK(cudaMemsetAsync(c->cntB.p, 0, sizeof(uint32_t) * (c->W + 1), s));
    launch_words(LA, s);
    exclusive_scan(c->cntA.p, c->cntA.p, c->W + 1, c->scan_tmp.p, s);
    exclusive_scan(c->cntB.p, c->cntB.p, c->W + 1, c->scan_tmp.p, s);
    CK(cudaGetLastError());
    uint32_t nA = 0, nB = 0;
    if (int r = read_u32(c, c->cntA.p + c->W, &nA)) return r;
    if (int r = read_u32(c, c->cntB.p + c->W, &nB)) return r;
    uint64_t nS64 = (uint64_t)nA + nB;
    if (nS64 >= 0xffffffe0ull) return fail(c, LBMDEM_ERR_INVALID_ARG, "lattice too large");
    uint32_t nS = (uint32_t)nS64;
    uint32_t nSpad = std::max<uint32_t>(32u, (nS + 31u) & ~31u);
    if ((uint64_t)Q * nSpad >= (1ull << 32))  // the kernels address populations with 32-bit offsets
        return fail(c, LBMDEM_ERR_INVALID_ARG, "lattice too large: %u stored nodes", nS);
    launch_words_bases(LA, nA, s);
    CK(c->coord.ensure(nSpad));
    CK(c->fbits.ensure(nSpad / 32));
    LA.coord = c->coord.p;
    launch_coords(LA, nA, nSpad, c->fbits.p, s);
    CK(cudaGetLastError());
    // populations
    const size_t esz = c->p.storage == LBMDEM_F32 ? 4 : 2;
    CK(c->f2.alloc((size_t)Q * nSpad * esz));
    CK(cudaMemsetAsync(c->f2.p, 0, esz * Q * nSpad, s));  // zero deviations: rest at rho_f
    Lat Lnew = make_lat(c);
    Lnew.nA = nA;
    Lnew.nS = nS;
    Lnew.nSpad = nSpad;
    Lnew.f = c->f2.p;
    Lnew.rec = c->rec2.p;
    Lnew.maskB = c->maskB2.p;
    if (!fresh && c->f.p) {
        Lat Lold = make_lat(c);
        launch_gather_old(Lnew, Lold, s);
        CK(cudaGetLastError());
    }
    c->f.swap(c->f2);
    c->f2.release();
    c->rec.swap(c->rec2);
    c->maskB.swap(c->maskB2);
    c->nA = nA;
    c->nS = nS;
    c->nSpad = nSpad;
    // band list and its candidate spheres
    CK(cudaMemsetAsync(c->band_count.p, 0, sizeof(uint32_t), s));
    CK(c->band_coord.ensure(1024));
    launch_band_collect(LA, c->band_coord.p, c->band_count.p, (uint32_t)c->band_coord.n, s);
    uint32_t nband = 0;
    if (int r = read_u32(c, c->band_count.p, &nband)) return r;
    if (nband > c->band_coord.n) {
        CK(c->band_coord.alloc(nband + nband / 8));
        CK(cudaMemsetAsync(c->band_count.p, 0, sizeof(uint32_t), s));
        launch_band_collect(LA, c->band_coord.p, c->band_count.p, (uint32_t)c->band_coord.n, s);
    }
    c->nband = nband;
    CK(c->band_cand.ensure(std::max<uint32_t>(nband, 1)));
    CK(c->band_slack.ensure(std::max<uint32_t>(nband, 1)));
    if (int r = build_cells(c)) return r;
    CellGrid Gb{};
    if (int r = build_cell_grid(c, Gb, c->Rmax + c->skin, c->band_cells)) return r;
    BandCand BC{c->Xref.p, c->Rd.p, c->skin, Gb, c->band_cells.start.p, c->band_cells.order.p,
                c->band_coord.p, c->band_cand.p, c->band_slack.p, nband, &c->st.p->status, c->band.p, nx, ny, nz};
    launch_band_cand(BC, s);
    CK(cudaGetLastError());
    if (nband > 0) {  // band ordered by slack
        CK(c->band_coord2.ensure(nband));
        CK(c->band_cand2.ensure(nband));
        CK(c->band_slack2.ensure(nband));
        CK(c->slack_hist.ensure(SLACK_HIST));
        launch_band_sort(c->band_coord.p, c->band_cand.p, c->band_slack.p, nband, c->skin, c->slack_hist.p,
                         c->scan_tmp.p, c->band_coord2.p, c->band_cand2.p, c->band_slack2.p, s);
        CK(cudaGetLastError());
        c->band_coord.swap(c->band_coord2);
        c->band_cand.swap(c->band_cand2);
        c->band_slack.swap(c->band_slack2);
    }
    // the owner map matches the layout positions only after the next map
    // update: it re-tests every band node, later ones skip nodes whose slack
    // exceeds the largest displacement since the layout
    CK(cudaMemsetAsync(&c->st.p->disp_layout_bits, 0, sizeof(uint32_t), s));
    CK(cudaMemsetAsync(&c->st.p->layout_fresh, 1, sizeof(uint32_t), s));
    // link lists, grouped by sphere (direction-major inside a sphere)
    int np = c->np;
    size_t ng = (size_t)std::max(np, 1) * LINK_GROUPS;
    CK(c->surf_count.ensure(ng + 2));  // + the total before padding
    CK(c->surf_off.ensure(ng + 1));
    CK(cudaMemsetAsync(c->surf_count.p, 0, sizeof(uint32_t) * (ng + 2), s));
    SurfArgs SA{};
    SA.L = make_lat(c);
    SA.X = c->Xref.p;
    SA.R = c->Rd.p;
    SA.reach_extra = c->skin + 1.5;
    SA.skin = c->skin;
    SA.owner = c->owner.p;
    SA.band = c->band.p;
    SA.count = c->surf_count.p;
    SA.nlink = c->surf_count.p + ng + 1;
    launch_surf_count(SA, np, s);
    exclusive_scan(c->surf_count.p, c->surf_off.p, ng + 1, c->scan_tmp.p, s);
    uint32_t nlink = 0;
    if (int r = read_u32(c, c->surf_off.p + ng, &nlink)) return r;
    if (int r = read_u32(c, c->surf_count.p + ng + 1, &c->nlink_raw)) return r;
    CK(c->surf_link.ensure(std::max<uint32_t>(nlink, 32)));
    CK(c->warp_p.ensure(std::max<uint32_t>(nlink / LINK_WARP, 1)));
    CK(c->chunk_dir.ensure(std::max<uint32_t>(nlink / 32, LINK_CHUNKS)));
    SA.offset = c->surf_off.p;
    SA.link = c->surf_link.p;
    SA.warp_p = c->warp_p.p;
    SA.chunk_dir = c->chunk_dir.p;
    launch_surf_fill(SA, np, s);
    CK(cudaGetLastError());
    c->nwarps = nlink / LINK_WARP;
    // even steps take their links inside the collide kernel (link words from
    // the owner map) unless the sphere indices do not fit a link word, or a
    // periodic axis is narrow enough for a link node (within R + sqrt(3) of a
    // centre, R + skin after motion) to neighbour two images of one sphere:
    // its links would need one lever per image, which the link lists keep
    const double reach = 2.0 * (c->Rmax + c->skin + 2.0);
    const bool wide = c->p.ny > reach && c->p.nz > reach && (!px || c->p.nx > reach);
    // (link_mode 0: with FP32 storage and spheres of radius 8 lu or more.
    // With 16-bit storage the even collide kernel is bandwidth-light, and
    // smaller spheres change along a 32-node run often enough that the
    // per-warp sphere sums cost more than the link kernel: R 5.7 FCC, 0.106
    // against 0.091 ms per step; R 11.4, 0.309 against 0.329 ms)
    const bool want = c->p.link_mode == 2 ||
                      (c->p.link_mode == 0 && c->p.storage == LBMDEM_F32 && c->Rmax >= 8.0);
    c->fused_links = want && c->nwarps > 0 && np <= LW_MAX_SPHERES && wide;
    if (c->fused_links) {
        CK(c->linkw.ensure(nSpad));
        launch_link_words(make_lat(c), c->linkw.p, s);
        CK(cudaGetLastError());
    }
    // conversion scratch
    uint32_t cap = c->p.max_flips > 0 ? (uint32_t)c->p.max_flips
                                      : std::min<uint32_t>(1u << 20, std::max<uint32_t>(4096u, nband / 8));
    if (cap != c->flip_cap) {
        CK(c->flip_rec.alloc(cap));
        CK(c->flip_scratch.alloc((size_t)cap * Q * Q));
        CK(c->flip_valid.alloc((size_t)cap * Q));
        c->flip_cap = cap;
    }
    // probe plane ranges in compact order
    c->pA0 = c->pA1 = c->pB0 = c->pB1 = 0;
    int xp = c->p.probe_x;
    if (xp >= 0 && xp < nx) {
        uint4 r0, r1;
        CK(cudaMemcpyAsync(&r0, c->rec.p + (size_t)xp * ny * c->nw, sizeof(uint4), cudaMemcpyDeviceToHost, s));
        if (xp + 1 < nx)
            CK(cudaMemcpyAsync(&r1, c->rec.p + (size_t)(xp + 1) * ny * c->nw, sizeof(uint4),
                               cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        c->pA0 = r0.z;
        c->pA1 = xp + 1 < nx ? r1.z : nA;
        c->pB0 = r0.w;
        c->pB1 = xp + 1 < nx ? r1.w : nS;
    }
    CK(cudaStreamSynchronize(s));
    destroy_graph(c);
    return 0;
}

// ------------------------------------------------------------ stepping

static void record_pair_begin(lbmdem_ctx* c, int group, size_t& idx, cudaStream_t st = nullptr) {
    if (!st) st = c->stream;
    idx = c->ev_pairs++;
    while (c->ev.size() < 2 * c->ev_pairs) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev.push_back(e);
    }
    if (c->ev_group.size() < c->ev_pairs) c->ev_group.resize(c->ev_pairs);
    c->ev_group[idx] = group;
    if (c->capturing)
        cudaEventRecordWithFlags(c->ev[2 * idx], st, cudaEventRecordExternal);
    else
        cudaEventRecord(c->ev[2 * idx], st);
}

static void record_pair_end(lbmdem_ctx* c, size_t idx, cudaStream_t st = nullptr) {
    if (!st) st = c->stream;
    if (c->capturing)
        cudaEventRecordWithFlags(c->ev[2 * idx + 1], st, cudaEventRecordExternal);
    else
        cudaEventRecord(c->ev[2 * idx + 1], st);
}

// kernels one step issues: map update (4 when there is a band, else 1),
// collide, links (if any surface entries and the step's links are not in the
// collide kernel), inlet/outlet (if any), DEM
static bool links_in_collide(const lbmdem_ctx* c, int parity) { return c->fused_links && parity == 0; }

static int64_t kernels_per_step(const lbmdem_ctx* c, int parity) {
    int64_t k = 1;  // DEM
    if (c->lbm) {
        k += c->nband ? 4 : 1;
        k += c->nS ? 1 : 0;
        k += c->nwarps && !links_in_collide(c, parity) ? 1 : 0;
        bool px = c->p.inlet == LBMDEM_X_PERIODIC;
        k += (!px && !(c->p.inlet != 0 && c->p.outlet > 1)) ? 1 : 0;
    }
    return k;
}

static bool inlet_outlet_active(const lbmdem_ctx* c) {
    return c->p.inlet != LBMDEM_X_PERIODIC && !(c->p.inlet != 0 && c->p.outlet > 1);
}

static void enqueue_step(lbmdem_ctx* c, int parity, bool monitor) {
    cudaStream_t s = c->stream;
    bool tm = c->timing;
    size_t e = 0;
    c->launches += kernels_per_step(c, parity);
    if (c->lbm) {
        Lat L = make_lat(c);
        PartView P = make_part(c);
        Band B{c->band_coord.p, c->band_cand.p, c->band_slack.p, c->nband};
        FlipBuf F{c->flip_rec.p, c->flip_scratch.p, c->flip_valid.p, c->flip_cap};
        if (tm) record_pair_begin(c, 2, e);
        launch_map_update(L, P, B, F, c->st.p, parity == 1, parity, c->fused_links ? c->linkw.p : nullptr, c->batched,
                          s);
        if (tm) record_pair_end(c, e);
        Mon mon{};
        DevStats* sd = c->st.p;
        mon.acc = sd->mon;
        mon.umax_bits = &sd->max_u_bits;
        mon.status = &sd->status;
        mon.probe_sum = c->p.probe_x >= 0 && !c->suppress_probe ? c->probe.p : nullptr;
        mon.t_dev = &sd->t;
        mon.pA0 = c->pA0;
        mon.pA1 = c->pA1;
        mon.pB0 = c->pB0;
        mon.pB1 = c->pB1;
        if (monitor) {
            cudaMemsetAsync(sd->mon, 0, sizeof(double) * 6, s);
            cudaMemsetAsync(&sd->max_u_bits, 0, sizeof(uint32_t), s);
        }
        const bool fused = links_in_collide(c, parity);
        if (tm) record_pair_begin(c, parity == 1 ? 0 : 5, e);
        if (fused)
            launch_collide_even_links(L, mon, P, c->linkw.p, monitor, c->p.tile > 0 ? c->p.tile : 64, s);
        else
            launch_collide(L, mon, parity == 1, monitor, c->p.tile > 0 ? c->p.tile : 64, s);
        if (tm) record_pair_end(c, e);
        if (!fused) {
            LinkLists LL{c->surf_link.p, c->warp_p.p, c->chunk_dir.p, c->nwarps};
            if (tm) record_pair_begin(c, 1, e);
            launch_links(L, P, LL, s);
            if (tm) record_pair_end(c, e);
        }
        // the inlet/outlet only needs this step's populations and the DEM only
        // this step's link sums: they run side by side, the boundary on a
        // side stream joined before the next step
        BC bc{c->p.inlet, c->p.outlet, c->src, &sd->t};
        if (inlet_outlet_active(c)) {
            cudaEventRecord(c->ev_fork, s);
            cudaStreamWaitEvent(c->side, c->ev_fork, 0);
            size_t e2 = 0;
            if (tm) record_pair_begin(c, 3, e2, c->side);
            launch_inlet_outlet(L, bc, parity == 0, c->side);
            if (tm) record_pair_end(c, e2, c->side);
            cudaEventRecord(c->ev_join, c->side);
            Dem D = make_dem(c);
            if (tm) record_pair_begin(c, 4, e);
            launch_dem_step(D, false, s);
            if (tm) record_pair_end(c, e);
            cudaStreamWaitEvent(s, c->ev_join, 0);
            return;
        }
    }
    Dem D = make_dem(c);
    if (tm) record_pair_begin(c, 4, e);
    launch_dem_step(D, false, s);
    if (tm) record_pair_end(c, e);
}

static int collect_timing(lbmdem_ctx* c) {
    if (c->ev_pairs == 0) return 0;
    CK(cudaStreamSynchronize(c->stream));
    for (size_t k = 0; k < c->ev_pairs; ++k) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->ev[2 * k], c->ev[2 * k + 1]));
        c->tm_ms[c->ev_group[k]] += ms;
        c->tm_n[c->ev_group[k]] += 1;
    }
    c->ev_pairs = 0;
    return 0;
}

static int ensure_probe(lbmdem_ctx* c, int64_t upto) {
    if (c->p.probe_x < 0) return 0;
    if ((size_t)upto <= c->probe_cap) return 0;
    size_t cap = std::max<size_t>((size_t)upto * 2, 4096);
    DBuf<double> nb;
    CK(nb.alloc(2 * cap));
    CK(cudaMemsetAsync(nb.p, 0, sizeof(double) * 2 * cap, c->stream));
    if (c->probe.p && c->probe_cap)
        CK(cudaMemcpyAsync(nb.p, c->probe.p, sizeof(double) * 2 * c->probe_cap, cudaMemcpyDeviceToDevice,
                           c->stream));
    c->probe.swap(nb);
    nb.release();
    c->probe_cap = cap;
    destroy_graph(c);
    return 0;
}

static int capture_graph(lbmdem_ctx* c) {
    destroy_graph(c);
    if (int r = collect_timing(c)) return r;
    bool mon = c->p.monitor_every > 0;
    int64_t l0 = c->launches;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    for (int k = 0; k < c->glen; ++k) enqueue_step(c, k & 1, mon && k == c->glen - 1);
    c->capturing = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess) return fail(c, LBMDEM_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(c, LBMDEM_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    c->gtiming = c->timing;
    // event pairs recorded during capture belong to the graph: they are
    // recorded again by every launch and read back after it
    c->glaunches = c->launches - l0;
    c->launches = l0;  // counted when the graph is launched
    c->gpairs = c->ev_pairs;
    c->gev_group.assign(c->ev_group.begin(), c->ev_group.begin() + c->gpairs);
    c->ev_pairs = 0;
    return 0;
}

static int relayout(lbmdem_ctx* c);

static int check_and_relayout(lbmdem_ctx* c, bool& did) {
    did = false;
    CK(cudaMemcpyAsync(c->st_host, c->st.p, sizeof(DevStats), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    int code = map_status(c->st_host->status);
    if (code) {
        c->status_latched = code;
        return fail(c, code, "%s", status_text(code));
    }
    float disp, vel;
    uint32_t db = c->st_host->max_disp_bits, vb = c->st_host->max_vel_bits;
    memcpy(&disp, &db, 4);
    memcpy(&vel, &vb, 4);
    CK(cudaMemsetAsync(&c->st.p->max_disp_bits, 0, 2 * sizeof(uint32_t), c->stream));
    if (disp > c->trigger && (c->t % 2) == 0) {
        if (int r = relayout(c)) return r;
        did = true;
        disp = 0.f;
    }
    // next check: before the fastest sphere could reach the trigger at twice
    // its current speed, and at least every 64 steps (spheres accelerate)
    double room = c->trigger - disp;
    double v = std::max<double>(vel, 1e-9);
    double steps = room > 0 ? room / (2.0 * v) : 1.0;
    c->steps_until_check = (int64_t)std::max(1.0, std::min(steps, 64.0));
    return 0;
}

// ------------------------------------------------------------ public API

static int relayout(lbmdem_ctx* c) {
    cudaStream_t s = c->stream;
    launch_rebase(c->Xref.p, c->dX.p, c->dXc.p, c->np, s);
    CK(cudaGetLastError());
    if (int r = build_cells(c)) return r;
    if (int r = build_neighbours(c, true)) return r;
    if (c->lbm) {
        if (int r = build_layout(c, false)) return r;
    }
    Dem D = make_dem(c);
    launch_dem_step(D, true, s);
    CK(cudaGetLastError());
    c->relayouts++;
    destroy_graph(c);
    return 0;
}

extern "C" {

void lbm_dem_default_params(lbmdem_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->nx = 64;
    p->ny = 16;
    p->nz = 16;
    p->tau = 0.8;
    p->rho_f = 1.0;
    p->storage = LBMDEM_F32;
    p->inlet = LBMDEM_INLET_PRESSURE;
    p->outlet = LBMDEM_OUT_ZERO_GRAD;
    p->dem_substeps = 10;
    p->E_p = 10.37;
    p->nu_p = 0.2;
    p->mu = 0.3;
    p->rho_p = 2.466;
    p->probe_x = -1;
    p->lbm_on = 1;
    p->skin = 0.0;
    p->dem_skin = 0.0;
    p->monitor_every = 0;
    p->graph_steps = 0;
    p->max_flips = 0;
    p->tile = 0;
    p->device = 0;
    p->link_mode = 0;
    p->cuda_stream = nullptr;
}

int lbm_dem_init(const lbmdem_params* pp, lbmdem_ctx** out) {
    lbmdem_ctx* c = nullptr;
    if (!out) return LBMDEM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!pp) return LBMDEM_ERR_INVALID_ARG;
    const lbmdem_params& p = *pp;
    if (p.nx < 1 || p.ny < 1 || p.nz < 1 || p.nx > 4096 || p.ny > 1024 || p.nz > 1024)
        return LBMDEM_ERR_INVALID_ARG;
    if (!(p.tau > 0.5) || !(p.rho_f > 0) || p.dem_substeps < 1) return LBMDEM_ERR_INVALID_ARG;
    if (p.storage != LBMDEM_F32 && p.storage != LBMDEM_BF16_DEV && p.storage != LBMDEM_F16_DEV)
        return LBMDEM_ERR_INVALID_ARG;
    if (p.inlet < 0 || p.inlet > 2 || p.outlet < 0 || p.outlet > 2) return LBMDEM_ERR_INVALID_ARG;
    if (p.inlet != LBMDEM_X_PERIODIC && p.nx < 3) return LBMDEM_ERR_INVALID_ARG;
    if (p.probe_x >= p.nx || p.probe_x < -1) return LBMDEM_ERR_INVALID_ARG;
    if (!(p.E_p > 0) || !(p.nu_p > -1 && p.nu_p < 0.5) || !(p.mu >= 0) || !(p.rho_p > 0))
        return LBMDEM_ERR_INVALID_ARG;
    if (p.tile != 0 && p.tile != 64 && p.tile != 128 && p.tile != 256) return LBMDEM_ERR_INVALID_ARG;
    if (p.link_mode < 0 || p.link_mode > 2) return LBMDEM_ERR_INVALID_ARG;
    if (p.skin < 0 || p.dem_skin < 0 || p.graph_steps < 0 || p.graph_steps % 2 || p.max_flips < 0)
        return LBMDEM_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= p.device || p.device < 0)
        return LBMDEM_ERR_NO_DEVICE;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, p.device) != cudaSuccess) return LBMDEM_ERR_NO_DEVICE;
    if (prop.major < 10) return LBMDEM_ERR_NO_DEVICE;
    c = new lbmdem_ctx();
    c->p = p;
    c->lbm = p.lbm_on != 0;
    c->skin = p.skin > 0 ? p.skin : 0.25;
    c->dem_skin = p.dem_skin > 0 ? p.dem_skin : 0.5;
    c->hard = std::min(c->skin, 0.5 * c->dem_skin);
    c->trigger = 0.5 * c->hard;
    c->glen = p.graph_steps > 0 ? p.graph_steps : 16;
    c->nw = (p.nz + 31) / 32;
    c->N = (size_t)p.nx * p.ny * p.nz;
    c->W = (size_t)p.nx * p.ny * c->nw;
    auto bail = [&](int code) {
        lbm_dem_destroy(c);
        return code;
    };
    if (cudaSetDevice(p.device) != cudaSuccess) return bail(LBMDEM_ERR_CUDA);
    if (p.cuda_stream) {
        c->stream = (cudaStream_t)p.cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(LBMDEM_ERR_CUDA);
        c->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return bail(LBMDEM_ERR_CUDA);
    if (c->st.alloc(1) != cudaSuccess) return bail(LBMDEM_ERR_OOM);
    if (cudaMallocHost((void**)&c->st_host, sizeof(DevStats)) != cudaSuccess) return bail(LBMDEM_ERR_OOM);
    if (cudaMemset(c->st.p, 0, sizeof(DevStats)) != cudaSuccess) return bail(LBMDEM_ERR_CUDA);
    if (c->lbm) {
        if (c->owner.alloc(c->N) || c->deep.alloc(c->N) || c->band.alloc(c->N) || c->rec.alloc(c->W) ||
            c->rec2.alloc(c->W) || c->maskB.alloc(c->W) || c->maskB2.alloc(c->W) ||
            c->cntA.alloc(c->W + 1) || c->cntB.alloc(c->W + 1) ||
            c->scan_tmp.alloc(scan_tmp_size(std::max(c->W + 1, (size_t)1 << 24))) ||
            c->band_count.alloc(1))
            return bail(LBMDEM_ERR_OOM);
    }
    c->src.waveform = LBMDEM_SINE;
    c->src.amp = 0.0;
    c->src.omega = 0.0;
    c->src.t0 = 0.0;
    c->src.t_n = -1;
    *out = c;
    return 0;
}

int lbm_dem_set_packing(lbmdem_ctx* c, int32_t n, const double* X, const double* Rh, const double* Vh,
                        const double* Wh, const uint8_t* fixedh) {
    if (!c) return LBMDEM_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!X || !Rh))) return fail(c, LBMDEM_ERR_INVALID_ARG, "bad packing arrays");
    CK(cudaSetDevice(c->p.device));
    const lbmdem_params& p = c->p;
    int px = p.inlet == LBMDEM_X_PERIODIC;
    double Rmax = 0, Rmin = 1e300;
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            if (!std::isfinite(X[3 * i + a])) return fail(c, LBMDEM_ERR_INVALID_ARG, "non-finite X[%d]", i);
            if (Vh && !std::isfinite(Vh[3 * i + a])) return fail(c, LBMDEM_ERR_INVALID_ARG, "non-finite V");
            if (Wh && !std::isfinite(Wh[3 * i + a])) return fail(c, LBMDEM_ERR_INVALID_ARG, "non-finite Omega");
        }
        if (!(Rh[i] > 0) || !std::isfinite(Rh[i])) return fail(c, LBMDEM_ERR_INVALID_ARG, "R[%d] <= 0", i);
        Rmax = std::max(Rmax, Rh[i]);
        Rmin = std::min(Rmin, Rh[i]);
    }
    // geometry limits: a node inside or within the skin of a sphere is so
    // for one image only (R + skin below half a periodic box; the link lists
    // then give each link the lever of its own image), and a sphere meets
    // each image of a neighbour through one neighbour entry
    if (c->lbm && Rmax + c->skin + 3.0 >= 127.0)
        return fail(c, LBMDEM_ERR_INVALID_ARG, "R + skin must stay below 124 lattice units");
    double lim_lbm = Rmax + c->skin;
    double lim_dem = 2 * Rmax + c->dem_skin;
    double Ls[3] = {(double)p.nx, (double)p.ny, (double)p.nz};
    for (int a = 0; a < 3; ++a) {
        bool per = a > 0 || px;
        if (!per || n == 0) continue;
        if (c->lbm && 2 * lim_lbm >= Ls[a])
            return fail(c, LBMDEM_ERR_INVALID_ARG, "R + skin must stay below half the periodic box (axis %d)", a);
        if (lim_dem > Ls[a])
            return fail(c, LBMDEM_ERR_INVALID_ARG, "2 R + dem_skin must not exceed the periodic box (axis %d)", a);
    }
    if (n > 0 && n <= 20000) {
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) {
                double d2 = 0;
                for (int a = 0; a < 3; ++a) {
                    double d = X[3 * j + a] - X[3 * i + a];
                    if (a > 0 || px) d -= Ls[a] * floor(d / Ls[a] + 0.5);
                    d2 += d * d;
                }
                double ov = Rh[i] + Rh[j] - sqrt(d2);
                if (ov >= std::min(Rh[i], Rh[j]))
                    return fail(c, LBMDEM_ERR_INVALID_ARG, "spheres %d and %d overlap by %.3g", i, j, ov);
            }
    }
    c->np = n;
    c->Rmax = Rmax;
    c->have_packing = false;
    destroy_graph(c);
    size_t nn = std::max(n, 1);
    CK(c->Xref.alloc(3 * nn));
    CK(c->Fh.alloc(3 * NREP * nn));
    CK(c->Th.alloc(3 * NREP * nn));
    CK(c->Fh_prev.alloc(3 * nn));
    CK(c->Th_prev.alloc(3 * nn));
    CK(c->Fa.alloc(nn));
    CK(c->Ta.alloc(nn));
    CK(c->dX.alloc(nn));
    CK(c->dXc.alloc(nn));
    CK(c->dXb.alloc(2 * nn));
    CK(c->V.alloc(nn));
    CK(c->Om.alloc(nn));
    CK(c->q.alloc(nn));
    CK(c->Vhb.alloc(2 * nn));
    CK(c->Whb.alloc(2 * nn));
    CK(c->Fc.alloc(nn));
    CK(c->Tc.alloc(nn));
    CK(c->xf.alloc(nn));
    CK(c->ab.alloc((Q - 1) * nn));
    CK(c->pk.alloc(3 * nn));
    CK(c->org.alloc(nn));
    CK(c->orgw.alloc(nn));
    CK(c->R.alloc(nn));
    CK(c->Rd.alloc(nn));
    CK(c->invm.alloc(nn));
    CK(c->invI.alloc(nn));
    CK(c->fixed.alloc(nn));
    // host staging of the per-sphere constants (marshalling only)
    std::vector<double> Xv(3 * nn, 0.0);
    std::vector<float4> Vv(nn), Wv(nn), qv(nn), zero4(nn);
    std::vector<float> Rv(nn, 1.f), imv(nn, 0.f), iIv(nn, 0.f);
    std::vector<double> Rdv(nn, 1.0);
    std::vector<uint8_t> fx(nn, 0);
    bool mobile = false;
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) Xv[3 * i + a] = X[3 * i + a];
        fx[i] = fixedh ? (fixedh[i] ? 1 : 0) : 0;
        float v[3] = {0, 0, 0}, w[3] = {0, 0, 0};
        if (!fx[i]) {
            mobile = true;
            for (int a = 0; a < 3; ++a) {
                v[a] = Vh ? (float)Vh[3 * i + a] : 0.f;
                w[a] = Wh ? (float)Wh[3 * i + a] : 0.f;
            }
        }
        Vv[i] = make_float4(v[0], v[1], v[2], 0.f);
        Wv[i] = make_float4(w[0], w[1], w[2], 0.f);
        qv[i] = make_float4(1.f, 0.f, 0.f, 0.f);
        double m = p.rho_p * 4.0 / 3.0 * M_PI * Rh[i] * Rh[i] * Rh[i];
        Rv[i] = (float)Rh[i];
        Rdv[i] = Rh[i];
        imv[i] = (float)(1.0 / m);
        iIv[i] = (float)(1.0 / (0.4 * m * Rh[i] * Rh[i]));
    }
    for (size_t i = 0; i < nn; ++i) zero4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    c->any_mobile = mobile;
    cudaStream_t s = c->stream;
    CK(cudaMemcpyAsync(c->Xref.p, Xv.data(), sizeof(double) * 3 * nn, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->V.p, Vv.data(), sizeof(float4) * nn, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->Om.p, Wv.data(), sizeof(float4) * nn, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->q.p, qv.data(), sizeof(float4) * nn, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->dX.p, zero4.data(), sizeof(float4) * nn, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->dXc.p, zero4.data(), sizeof(float4) * nn, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->R.p, Rv.data(), sizeof(float) * nn, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->Rd.p, Rdv.data(), sizeof(double) * nn, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->invm.p, imv.data(), sizeof(float) * nn, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->invI.p, iIv.data(), sizeof(float) * nn, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->fixed.p, fx.data(), nn, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(c->Fh.p, 0, sizeof(double) * 3 * NREP * nn, s));
    CK(cudaMemsetAsync(c->Th.p, 0, sizeof(double) * 3 * NREP * nn, s));
    CK(cudaMemsetAsync(c->Fh_prev.p, 0, sizeof(double) * 3 * nn, s));
    CK(cudaMemsetAsync(c->Th_prev.p, 0, sizeof(double) * 3 * nn, s));
    CK(cudaMemsetAsync(c->st.p, 0, sizeof(DevStats), s));
    if (int r = build_cells(c)) return r;
    if (int r = build_neighbours(c, false)) return r;
    if (c->lbm) {
        if (int r = build_layout(c, true)) return r;
    }
    c->t = 0;
    c->mon_step = -1;
    c->probe_cap = 0;
    c->probe.release();
    if (int r = ensure_probe(c, 4096)) return r;
    Dem D = make_dem(c);
    launch_dem_step(D, true, s);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(c->st_host, c->st.p, sizeof(DevStats), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int code = map_status(c->st_host->status);
    if (code) {
        c->status_latched = code;
        return fail(c, code, "set_packing: %s", status_text(code));
    }
    c->status_latched = 0;
    c->steps_until_check = 0;
    c->have_packing = true;
    c->err.clear();
    return 0;
}

int lbm_dem_set_pressure_source(lbmdem_ctx* c, int32_t waveform, double amplitude, double omega,
                                int64_t t_n, double t0) {
    if (!c) return LBMDEM_ERR_INVALID_ARG;
    if (waveform < 0 || waveform > LBMDEM_RICKER || !std::isfinite(amplitude) || !std::isfinite(omega) ||
        !std::isfinite(t0))
        return fail(c, LBMDEM_ERR_INVALID_ARG, "bad source");
    c->src.waveform = waveform;
    c->src.amp = amplitude;
    c->src.omega = omega;
    c->src.t_n = t_n;
    c->src.t0 = t0;
    destroy_graph(c);
    return 0;
}

int lbm_dem_step(lbmdem_ctx* c, int64_t n) {
    if (!c) return LBMDEM_ERR_INVALID_ARG;
    if (n < 0) return fail(c, LBMDEM_ERR_INVALID_ARG, "n < 0");
    if (!c->have_packing) return fail(c, LBMDEM_ERR_STATE, "step before set_packing");
    if (c->status_latched) return fail(c, c->status_latched, "%s", status_text(c->status_latched));
    CK(cudaSetDevice(c->p.device));
    if (int r = ensure_probe(c, c->t + n + 1)) return r;
    bool checks = c->any_mobile;
    while (n > 0) {
        if (checks && c->steps_until_check <= 0) {
            bool did;
            if (int r = check_and_relayout(c, did)) return r;
        }
        int64_t room = checks ? c->steps_until_check : n;
        bool use_graph = (c->t % 2 == 0) && n >= c->glen && room >= c->glen;
        if (use_graph) {
            if (!c->gexec || c->gtiming != c->timing) {
                if (int r = capture_graph(c)) return r;
            }
            CK(cudaGraphLaunch(c->gexec, c->stream));
            c->launches += c->glaunches;
            if (c->p.monitor_every > 0) c->mon_step = c->t + c->glen - 1;
            c->t += c->glen;
            n -= c->glen;
            c->steps_until_check -= c->glen;
            if (c->timing) {
                c->ev_pairs = c->gpairs;
                for (size_t k = 0; k < c->gpairs; ++k) c->ev_group[k] = c->gev_group[k];
                if (int r = collect_timing(c)) return r;
            }
        } else {
            bool mon = c->p.monitor_every > 0 && ((c->t + 1) % c->p.monitor_every == 0);
            size_t pairs0 = c->ev_pairs;
            enqueue_step(c, (int)(c->t & 1), mon);
            CK(cudaGetLastError());
            if (mon) c->mon_step = c->t;
            c->t += 1;
            n -= 1;
            c->steps_until_check -= 1;
            if (c->timing && c->ev_pairs > pairs0) {
                if (int r = collect_timing(c)) return r;
            }
        }
    }
    return 0;
}

// ------------------------------------------------------------ batched columns

}  // extern "C"

// A batch advances several independent contexts (columns) of one device
// together, each by its own number of steps, in ONE launch of one CUDA
// graph: every column is a parallel branch holding a device-side WHILE
// loop (a conditional graph node) whose body is two coupled steps of that
// column (an even and an odd one, so the AA parity of the captured kernels
// never changes) followed by a control kernel; an IF node after the loop
// takes a trailing single step when the column's count is odd.  The
// control kernel counts the column's remaining step pairs down and ends the
// loop when they run out, when the column's device status latched an error
// (NaN, capacity, skin) or when the batch's time limit has passed on the
// GPU clock (%globaltimer), in which case it latches LBMDEM_ERR_TIMEOUT: no
// loop runs unbounded, and nothing waits on another block.  The host takes
// no part until the whole sweep has run: re-layout checks happen before the
// launch only, so a sphere that moves farther than the skin inside the
// launch latches LBMDEM_ERR_SKIN instead.
struct lbmdem_batch {
    std::vector<lbmdem_ctx*> cols;
    int device = 0;
    cudaStream_t master = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<cudaEvent_t> pre;
    cudaGraphExec_t gexec = nullptr;
    DBuf<long long> remaining;         // [n] step pairs left per column (device)
    DBuf<long long> pairs_dev;         // [n] pair counts the start node reads
    DBuf<unsigned long long> start_ns; // GPU clock at the launch (device)
    double time_limit_s = 0.0;         // 0: no limit
    int64_t graph_launches = 0;        // graph launches so far
    std::vector<int64_t> requested;    // steps asked of each column by the last launch
    std::string err;
};

namespace {
int bfail(lbmdem_batch* b, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    return code;
}

#define BCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return bfail(b, LBMDEM_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),      \
                         __FILE__, __LINE__);                                                      \
    } while (0)

__device__ __forceinline__ unsigned long long gpu_clock_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct BatchCtl {
    long long* remaining;
    unsigned long long* start_ns;
    unsigned long long limit_ns;  // 0: none
};

// at the launch: the GPU clock and every column's pair count
__global__ void k_batch_start(BatchCtl ctl, const long long* pairs, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *ctl.start_ns = gpu_clock_ns();
    if (i < n) ctl.remaining[i] = pairs[i];
}

// end of one loop iteration (two steps) of column i: continue while pairs
// are left, the column's status is clear and the time limit has not passed
__global__ void k_batch_loop(BatchCtl ctl, int i, uint32_t* status, cudaGraphConditionalHandle h) {
    if (threadIdx.x || blockIdx.x) return;
    const long long r = ctl.remaining[i] - 1;
    ctl.remaining[i] = r;
    unsigned go = r > 0 && *status == 0u;
    if (go && ctl.limit_ns && gpu_clock_ns() - *ctl.start_ns > ctl.limit_ns) {
        atomicOr(status, ST_TIMEOUT);
        go = 0;
    }
    cudaGraphSetConditional(h, go);
}

// after the loop of a column with an odd step count: the trailing step runs
// only if the loop ran to its end with a clear status and time remains
__global__ void k_batch_tail(BatchCtl ctl, int i, uint32_t* status, cudaGraphConditionalHandle h) {
    if (threadIdx.x || blockIdx.x) return;
    unsigned go = ctl.remaining[i] <= 0 && *status == 0u;
    if (go && ctl.limit_ns && gpu_clock_ns() - *ctl.start_ns > ctl.limit_ns) {
        atomicOr(status, ST_TIMEOUT);
        go = 0;
    }
    cudaGraphSetConditional(h, go);
}

void batch_destroy_graph(lbmdem_batch* b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
}

// a conditional node (WHILE or IF) on `graph` after `dep`; its body graph
// is returned in *body
int add_conditional(lbmdem_batch* b, cudaGraph_t graph, cudaGraphNode_t dep, cudaGraphConditionalNodeType type,
                    cudaGraphConditionalHandle h, cudaGraphNode_t* node, cudaGraph_t* body) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = type;
    cp.conditional.size = 1;
    BCK(cudaGraphAddNode(node, graph, &dep, nullptr, 1, &cp));
    *body = cp.conditional.phGraph_out[0];
    return 0;
}

// capture `nsteps` coupled steps of column c (parities 0, 1, ...) and then
// the control kernel `ctl_kernel` into `body`
int capture_body(lbmdem_batch* b, lbmdem_ctx* c, cudaGraph_t body, int nsteps, void (*ctl_kernel)(BatchCtl, int, uint32_t*, cudaGraphConditionalHandle),
                 const BatchCtl& ctl, int i, cudaGraphConditionalHandle h) {
    BCK(cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const bool mon = c->p.monitor_every > 0;
    c->batched = true;
    for (int k = 0; k < nsteps; ++k) enqueue_step(c, k & 1, mon && k == nsteps - 1);
    c->batched = false;
    if (ctl_kernel) ctl_kernel<<<1, 32, 0, c->stream>>>(ctl, i, &c->st.p->status, h);
    cudaGraph_t g = body;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess) return bfail(b, LBMDEM_ERR_CUDA, "batch body capture: %s", cudaGetErrorString(e));
    return 0;
}

// One graph for the whole run: per column a WHILE loop over step pairs and,
// for an odd count, an IF node with the last step.
int batch_build(lbmdem_batch* b, const std::vector<int64_t>& steps) {
    batch_destroy_graph(b);
    const int n = (int)b->cols.size();
    std::vector<long long> pairs(n);
    for (int i = 0; i < n; ++i) pairs[i] = steps[i] / 2;
    DBuf<long long> dpairs;
    BCK(dpairs.alloc(n));
    BCK(cudaMemcpy(dpairs.p, pairs.data(), sizeof(long long) * n, cudaMemcpyHostToDevice));
    BatchCtl ctl{b->remaining.p, b->start_ns.p,
                 b->time_limit_s > 0 ? (unsigned long long)(b->time_limit_s * 1e9) + 1ull : 0ull};
    cudaGraph_t root = nullptr;
    BCK(cudaGraphCreate(&root, 0));
    auto bail = [&](int r) {
        cudaGraphDestroy(root);
        return r;
    };
    // the start node: a kernel node reading the pair counts (kept alive by
    // the graph's copy of the parameters; the buffer is re-made per build)
    cudaKernelNodeParams kp = {};
    void* args[3];
    long long* pp = dpairs.p;
    args[0] = &ctl;
    args[1] = &pp;
    args[2] = (void*)&n;
    kp.func = (void*)k_batch_start;
    kp.gridDim = dim3((unsigned)((n + 127) / 128), 1, 1);
    kp.blockDim = dim3(128, 1, 1);
    kp.kernelParams = args;
    cudaGraphNode_t start = nullptr;
    if (cudaGraphAddKernelNode(&start, root, nullptr, 0, &kp) != cudaSuccess)
        return bail(bfail(b, LBMDEM_ERR_CUDA, "batch: start node"));
    for (int i = 0; i < n; ++i) {
        lbmdem_ctx* c = b->cols[i];
        if (steps[i] <= 0) continue;
        const bool tm = c->timing;
        c->timing = false;  // per-kernel timing is not recorded inside a batch
        const int64_t l0 = c->launches;
        cudaGraphNode_t last = start;
        if (pairs[i] > 0) {
            cudaGraphConditionalHandle h;
            if (cudaGraphConditionalHandleCreate(&h, root, 1u, cudaGraphCondAssignDefault) != cudaSuccess)
                return bail(bfail(b, LBMDEM_ERR_CUDA, "batch: loop handle"));
            cudaGraph_t body;
            if (int r = add_conditional(b, root, start, cudaGraphCondTypeWhile, h, &last, &body)) return bail(r);
            if (int r = capture_body(b, c, body, 2, k_batch_loop, ctl, i, h)) return bail(r);
        }
        if (steps[i] % 2) {
            cudaGraphConditionalHandle h;
            if (cudaGraphConditionalHandleCreate(&h, root, 0u, cudaGraphCondAssignDefault) != cudaSuccess)
                return bail(bfail(b, LBMDEM_ERR_CUDA, "batch: tail handle"));
            // the decision kernel, then the IF node with one even step
            cudaKernelNodeParams tp = {};
            int ii = i;
            uint32_t* st = &c->st.p->status;
            void* targs[4] = {&ctl, &ii, &st, &h};
            tp.func = (void*)k_batch_tail;
            tp.gridDim = dim3(1, 1, 1);
            tp.blockDim = dim3(32, 1, 1);
            tp.kernelParams = targs;
            cudaGraphNode_t dec = nullptr;
            if (cudaGraphAddKernelNode(&dec, root, &last, 1, &tp) != cudaSuccess)
                return bail(bfail(b, LBMDEM_ERR_CUDA, "batch: tail decision node"));
            cudaGraph_t body;
            if (int r = add_conditional(b, root, dec, cudaGraphCondTypeIf, h, &last, &body)) return bail(r);
            if (int r = capture_body(b, c, body, 1, nullptr, ctl, i, h)) return bail(r);
        }
        c->launches = l0;  // counted per step when the graph runs
        c->timing = tm;
    }
    cudaError_t e = cudaGraphInstantiate(&b->gexec, root, 0);
    cudaGraphDestroy(root);
    if (e != cudaSuccess) return bfail(b, LBMDEM_ERR_CUDA, "batch instantiate: %s", cudaGetErrorString(e));
    // the pair counts are read by the start node at every launch: keep them
    dpairs.swap(b->pairs_dev);
    return 0;
}
}  // namespace

extern "C" {

int lbm_dem_batch_create(lbmdem_ctx* const* cols, int32_t n, lbmdem_batch** out) {
    if (!out) return LBMDEM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cols || n <= 0) return LBMDEM_ERR_INVALID_ARG;
    int dev = -1;
    for (int i = 0; i < n; ++i) {
        if (!cols[i]) return LBMDEM_ERR_INVALID_ARG;
        if (!cols[i]->have_packing) return LBMDEM_ERR_STATE;
        for (int j = 0; j < i; ++j)
            if (cols[j] == cols[i]) return LBMDEM_ERR_INVALID_ARG;
        if (dev >= 0 && cols[i]->p.device != dev) return LBMDEM_ERR_INVALID_ARG;
        dev = cols[i]->p.device;
    }
    lbmdem_batch* b = new lbmdem_batch();
    b->cols.assign(cols, cols + n);
    b->device = dev;
    if (cudaSetDevice(dev) != cudaSuccess || cudaStreamCreateWithFlags(&b->master, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess ||
        b->remaining.alloc(n) != cudaSuccess || b->start_ns.alloc(1) != cudaSuccess) {
        lbm_dem_batch_destroy(b);
        return LBMDEM_ERR_CUDA;
    }
    b->pre.resize(n, nullptr);
    for (int i = 0; i < n; ++i)
        if (cudaEventCreateWithFlags(&b->pre[i], cudaEventDisableTiming) != cudaSuccess) {
            lbm_dem_batch_destroy(b);
            return LBMDEM_ERR_CUDA;
        }
    *out = b;
    return 0;
}

int lbm_dem_batch_set_time_limit(lbmdem_batch* b, double seconds) {
    if (!b || !(seconds >= 0) || !std::isfinite(seconds)) return LBMDEM_ERR_INVALID_ARG;
    b->time_limit_s = seconds;
    batch_destroy_graph(b);
    return 0;
}

int lbm_dem_batch_step(lbmdem_batch* b, const int64_t* steps) {
    if (!b || !steps) return LBMDEM_ERR_INVALID_ARG;
    const int n = (int)b->cols.size();
    BCK(cudaSetDevice(b->device));
    std::vector<int64_t> rem(steps, steps + n);
    for (int i = 0; i < n; ++i) {
        lbmdem_ctx* c = b->cols[i];
        if (rem[i] < 0) return bfail(b, LBMDEM_ERR_INVALID_ARG, "steps[%d] < 0", i);
        if (c->status_latched)
            return bfail(b, c->status_latched, "column %d: %s", i, status_text(c->status_latched));
        if (int r = ensure_probe(c, c->t + rem[i] + 1)) return bfail(b, r, "column %d: %s", i, c->err.c_str());
        if (rem[i] == 0) continue;
        // host-side work before the launch: the re-layout decision, and a
        // single step to reach an even step count (the loops start even)
        if (c->any_mobile) {
            bool did;
            if (int r = check_and_relayout(c, did)) return bfail(b, r, "column %d: %s", i, c->err.c_str());
        }
        if (c->t % 2) {
            if (int r = lbm_dem_step(c, 1)) return bfail(b, r, "column %d: %s", i, c->err.c_str());
            rem[i] -= 1;
        }
    }
    // the graph holds the columns' device pointers and source parameters,
    // which set_packing, re-layouts and source changes replace: built anew
    // for every call (instantiation takes milliseconds, a sweep seconds)
    if (int r = batch_build(b, rem)) return r;
    b->requested = rem;
    for (int i = 0; i < n; ++i) {  // the graph runs after each column's earlier work
        BCK(cudaEventRecord(b->pre[i], b->cols[i]->stream));
        BCK(cudaStreamWaitEvent(b->master, b->pre[i], 0));
    }
    BCK(cudaGraphLaunch(b->gexec, b->master));
    b->graph_launches += 1;
    BCK(cudaEventRecord(b->done, b->master));
    for (int i = 0; i < n; ++i) {  // and before each column's later work
        lbmdem_ctx* c = b->cols[i];
        BCK(cudaStreamWaitEvent(c->stream, b->done, 0));
        if (rem[i] <= 0) continue;
        for (int64_t k = 0; k < rem[i]; ++k) c->launches += kernels_per_step(c, (int)((c->t + k) & 1));
        c->launches += (rem[i] + 1) / 2;  // loop control
        if (c->p.monitor_every > 0) c->mon_step = c->t + rem[i] - 1;
        c->t += rem[i];  // corrected from the device count by lbm_dem_batch_sync if a loop stopped early
        c->steps_until_check = 0;
    }
    return 0;
}

int lbm_dem_batch_sync(lbmdem_batch* b) {
    if (!b) return LBMDEM_ERR_INVALID_ARG;
    BCK(cudaSetDevice(b->device));
    BCK(cudaStreamSynchronize(b->master));
    int first = 0;
    for (lbmdem_ctx* c : b->cols) {
        int r = lbm_dem_status(c);
        // the device counts every step begun: a loop that stopped early
        // (latched status, time limit) leaves the context at that count
        if (r && c->lbm) c->t = (int64_t)c->st_host->t;
        if (r && !first) {
            first = r;
            bfail(b, r, "%s", c->err.empty() ? status_text(r) : c->err.c_str());
        }
    }
    return first;
}

int64_t lbm_dem_batch_graph_launches(const lbmdem_batch* b) { return b ? b->graph_launches : -1; }

const char* lbm_dem_batch_last_error(const lbmdem_batch* b) { return b ? b->err.c_str() : "null batch"; }

void lbm_dem_batch_destroy(lbmdem_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->master) cudaStreamSynchronize(b->master);
    batch_destroy_graph(b);
    for (cudaEvent_t e : b->pre)
        if (e) cudaEventDestroy(e);
    if (b->done) cudaEventDestroy(b->done);
    if (b->master) cudaStreamDestroy(b->master);
    delete b;
}

// ------------------------------------------------------------ adjoint

}  // extern "C"

namespace {
// shape(t) of the source, rho_in = rho_f + amplitude * shape(t) (Eq. 25,
// Table 2; Ricker: a = pi f (t - t0), f = omega / 2 pi)
double source_shape(const Source& S, int64_t t) {
    if (S.t_n >= 0 && t > S.t_n) return 0.0;
    double ph = S.omega * (double)t;
    switch (S.waveform) {
        case LBMDEM_SINE: return std::sin(ph);
        case LBMDEM_COSINE: return 1.0 - std::cos(ph);
        case LBMDEM_STEP: return 1.0;
        case LBMDEM_RICKER: {
            double a = 0.5 * S.omega * ((double)t - S.t0);
            return (1.0 - 2.0 * a * a) * std::exp(-a * a);
        }
    }
    return 0.0;
}
}  // namespace

extern "C" {

int lbm_dem_adjoint(lbmdem_ctx* c, int64_t steps, int32_t every, const double* target, double* loss,
                    double* dL_dtau, double* dL_damp, double* trace_out) {
    if (!c || steps <= 0 || !target || every < 2 || every % 2) return fail(c, LBMDEM_ERR_INVALID_ARG, "adjoint: arguments");
    if (!c->have_packing || !c->lbm) return fail(c, LBMDEM_ERR_STATE, "adjoint: needs a packing and the fluid");
    if (c->any_mobile) return fail(c, LBMDEM_ERR_STATE, "adjoint: every sphere must be fixed");
    if (c->p.probe_x < 0) return fail(c, LBMDEM_ERR_STATE, "adjoint: no probe plane");
    if (c->t % 2) return fail(c, LBMDEM_ERR_STATE, "adjoint: needs an even step count");
    if (c->status_latched) return fail(c, c->status_latched, "%s", status_text(c->status_latched));
    CK(cudaSetDevice(c->p.device));
    cudaStream_t s = c->stream;
    const int64_t t0 = c->t;
    const size_t esz = c->p.storage == LBMDEM_F32 ? 4 : 2;
    const size_t fbytes = (size_t)Q * c->nSpad * esz;
    const int64_t nseg = (steps + every - 1) / every;
    // forward with a checkpoint of the populations at the start of every segment
    DBuf<uint8_t> ck;
    CK(ck.alloc(fbytes * (size_t)nseg));
    for (int64_t g = 0; g < nseg; ++g) {
        CK(cudaMemcpyAsync(ck.p + fbytes * g, c->f.p, fbytes, cudaMemcpyDeviceToDevice, s));
        int64_t n = std::min<int64_t>(every, steps - g * every);
        if (int r = lbm_dem_step(c, n)) return r;
    }
    std::vector<double> trace((size_t)(t0 + steps));
    int64_t len = 0;
    if (int r = lbm_dem_read_probe(c, trace.data(), t0 + steps, &len)) return r;
    // loss and its derivative: p = c_s^2 rho (probe-plane mean)
    const double cs2 = 1.0 / 3.0;
    std::vector<double> dl((size_t)steps);
    double L = 0.0;
    for (int64_t k = 0; k < steps; ++k) {
        double p = cs2 * trace[(size_t)(t0 + k)], e = p - target[k];
        L += e * e;
        dl[(size_t)k] = 2.0 * e;
        if (trace_out) trace_out[k] = p;
    }
    // probe-plane fluid nodes (static: every sphere is fixed)
    int64_t np_plane = 0;
    {
        std::vector<uint32_t> fb(c->nSpad / 32), coord(c->nSpad);
        CK(cudaMemcpy(fb.data(), c->fbits.p, sizeof(uint32_t) * fb.size(), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(coord.data(), c->coord.p, sizeof(uint32_t) * coord.size(), cudaMemcpyDeviceToHost));
        for (uint32_t i = 0; i < c->nS; ++i)
            if ((fb[i >> 5] >> (i & 31) & 1u) && (int)(coord[i] >> 20) == c->p.probe_x) ++np_plane;
    }
    if (np_plane == 0) return fail(c, LBMDEM_ERR_STATE, "adjoint: probe plane without fluid");
    // backward: recompute each segment from its checkpoint, keeping the
    // natural populations of every step, then walk the adjoint back
    const size_t nbytes = (size_t)Q * c->nSpad * sizeof(float);
    DBuf<float> nat, adj, adj2;
    DBuf<uint32_t> nbr;
    DBuf<double> grads;
    CK(nat.alloc((size_t)Q * c->nSpad * (size_t)every));
    CK(adj.alloc((size_t)Q * c->nSpad));
    CK(adj2.alloc((size_t)Q * c->nSpad));
    CK(nbr.alloc((size_t)(Q - 1) * c->nSpad));
    CK(grads.alloc(GRAD_COPIES + 1));  // omega derivative copies, then the amplitude's
    CK(cudaMemsetAsync(adj.p, 0, nbytes, s));
    CK(cudaMemsetAsync(grads.p, 0, (GRAD_COPIES + 1) * sizeof(double), s));
    launch_adj_nbr(make_lat(c), nbr.p, s);
    CK(cudaGetLastError());
    const int64_t t_end = c->t;
    for (int64_t g = nseg - 1; g >= 0; --g) {
        int64_t n = std::min<int64_t>(every, steps - g * every);
        int64_t tg = t0 + g * every;
        CK(cudaMemcpyAsync(c->f.p, ck.p + fbytes * g, fbytes, cudaMemcpyDeviceToDevice, s));
        unsigned long long tdev = (unsigned long long)tg;
        CK(cudaMemcpyAsync(&c->st.p->t, &tdev, sizeof(tdev), cudaMemcpyHostToDevice, s));
        c->t = tg;
        Lat L = make_lat(c);
        for (int64_t k = 0; k < n; ++k) {
            launch_adj_snapshot(L, (c->t & 1) == 1, nat.p + (size_t)Q * c->nSpad * k, s);
            c->suppress_probe = true;  // the trace is already complete
            enqueue_step(c, (int)(c->t & 1), false);
            c->suppress_probe = false;
            c->t += 1;
        }
        CK(cudaGetLastError());
        AdjArgs A{L, nbr.p, adj.p, c->p.inlet, c->p.outlet, c->p.probe_x};
        for (int64_t k = n - 1; k >= 0; --k) {
            int64_t t = tg + k;  // step t -> t + 1
            A.adj = adj.p;
            launch_adj_boundary(A, source_shape(c->src, t + 1), grads.p + GRAD_COPIES, s);
            float dlt = (float)(dl[(size_t)(t - t0)] * cs2 / (double)np_plane);
            launch_adj_step(A, nat.p + (size_t)Q * c->nSpad * k, adj2.p, dlt, grads.p, s);
            adj.swap(adj2);
        }
        CK(cudaGetLastError());
    }
    // leave the context where the forward run ended
    c->t = t_end;
    {
        // the last segment's recomputation ended at t_end with the same state
        unsigned long long tdev = (unsigned long long)t_end;
        CK(cudaMemcpyAsync(&c->st.p->t, &tdev, sizeof(tdev), cudaMemcpyHostToDevice, s));
    }
    double gh[GRAD_COPIES + 1];
    CK(cudaMemcpyAsync(gh, grads.p, sizeof(gh), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double d_omega = 0.0;
    for (int k = 0; k < GRAD_COPIES; ++k) d_omega += gh[k];
    if (loss) *loss = L;
    const double om = 1.0 / c->p.tau;
    if (dL_dtau) *dL_dtau = -om * om * d_omega;  // d omega / d tau = -1 / tau^2
    if (dL_damp) *dL_damp = gh[GRAD_COPIES];
    return lbm_dem_status(c);
}

__global__ void k_centres(Dem D, double* X) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D.n) return;
    float4 d = D.dX[i], c = D.dXc[i];
    X[3 * i] = D.Xref[3 * i] + (double)d.x - (double)c.x;
    X[3 * i + 1] = D.Xref[3 * i + 1] + (double)d.y - (double)c.y;
    X[3 * i + 2] = D.Xref[3 * i + 2] + (double)d.z - (double)c.z;
}

int lbm_dem_adjoint_psm(lbmdem_ctx* c, int64_t steps, int32_t every, const double* target, double* loss,
                        double* dL_dtau, double* dL_damp, double* dL_dX, double* trace_out) {
    if (!c || steps <= 0 || !target || every < 1) return fail(c, LBMDEM_ERR_INVALID_ARG, "adjoint_psm: arguments");
    if (!c->have_packing || !c->lbm) return fail(c, LBMDEM_ERR_STATE, "adjoint_psm: needs a packing and the fluid");
    if (c->any_mobile) return fail(c, LBMDEM_ERR_STATE, "adjoint_psm: every sphere must be fixed");
    if (c->p.probe_x < 0) return fail(c, LBMDEM_ERR_STATE, "adjoint_psm: no probe plane");
    if (c->p.inlet == LBMDEM_X_WALL) return fail(c, LBMDEM_ERR_STATE, "adjoint_psm: needs a pressure inlet or periodic x");
    CK(cudaSetDevice(c->p.device));
    cudaStream_t s = c->stream;
    const size_t N = c->N, QN = (size_t)Q * N;
    PsmArgs A{c->p.nx, c->p.ny, c->p.nz, c->p.inlet == LBMDEM_X_PERIODIC, c->p.inlet, c->p.outlet, c->p.probe_x,
              (float)c->p.rho_f, (float)c->p.tau, N};
    const int64_t nseg = (steps + every - 1) / every;
    const int n = c->np;
    DBuf<float> g0, g1, eps, lam0, lam1, ck, snap;
    DBuf<double> X, trace, grads, G, dX;
    CK(g0.alloc(QN));
    CK(g1.alloc(QN));
    CK(eps.alloc(N));
    const bool grads_wanted = dL_dtau || dL_damp || dL_dX;
    CK(ck.alloc(grads_wanted ? QN * (size_t)nseg : 1));
    CK(snap.alloc(grads_wanted ? QN * (size_t)every : 1));
    CK(X.alloc(3 * (size_t)std::max(n, 1)));
    CK(trace.alloc((size_t)steps));
    CK(grads.alloc(GRAD_COPIES + 1));  // tau derivative copies, then the amplitude's
    CK(G.alloc(N));
    CK(dX.alloc(3 * (size_t)std::max(n, 1)));
    // the surrogate starts from rest at rho_f, source time 0
    CK(cudaMemsetAsync(g0.p, 0, sizeof(float) * QN, s));
    CK(cudaMemsetAsync(trace.p, 0, sizeof(double) * steps, s));
    CK(cudaMemsetAsync(grads.p, 0, (GRAD_COPIES + 1) * sizeof(double), s));
    CK(cudaMemsetAsync(G.p, 0, sizeof(double) * N, s));
    if (n > 0) {
        k_centres<<<(n + 127) / 128, 128, 0, s>>>(make_dem(c), X.p);
        CK(cudaGetLastError());
    }
    launch_psm_eps(A, X.p, c->Rd.p, n, eps.p, s);
    CK(cudaGetLastError());
    // forward with a checkpoint at the start of every segment
    for (int64_t t = 0; t < steps; ++t) {
        if (grads_wanted && t % every == 0)
            CK(cudaMemcpyAsync(ck.p + QN * (size_t)(t / every), g0.p, sizeof(float) * QN, cudaMemcpyDeviceToDevice, s));
        launch_psm_probe(A, g0.p, trace.p + t, s);
        launch_psm_step(A, g0.p, g1.p, eps.p, s);
        launch_psm_boundary(A, g1.p, c->src, (unsigned long long)(t + 1), s);
        g0.swap(g1);
    }
    CK(cudaGetLastError());
    std::vector<double> tr((size_t)steps);
    CK(cudaMemcpyAsync(tr.data(), trace.p, sizeof(double) * steps, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double cs2 = 1.0 / 3.0, nplane = (double)c->p.ny * c->p.nz;
    std::vector<double> dl((size_t)steps);
    double L = 0.0;
    for (int64_t k = 0; k < steps; ++k) {
        const double p = cs2 * (c->p.rho_f + tr[(size_t)k] / nplane), e = p - target[k];
        L += e * e;
        dl[(size_t)k] = 2.0 * e * cs2 / nplane;
        if (trace_out) trace_out[k] = p;
    }
    if (loss) *loss = L;
    if (!dL_dtau && !dL_damp && !dL_dX) return lbm_dem_status(c);  // the forward loss alone
    // backward: recompute each segment from its checkpoint, then the adjoint
    CK(lam0.alloc(QN));
    CK(lam1.alloc(QN));
    CK(cudaMemsetAsync(lam0.p, 0, sizeof(float) * QN, s));
    for (int64_t seg = nseg - 1; seg >= 0; --seg) {
        const int64_t tg = seg * every, m = std::min<int64_t>(every, steps - tg);
        // the recomputed states go straight into their snapshot slots
        CK(cudaMemcpyAsync(snap.p, ck.p + QN * (size_t)seg, sizeof(float) * QN, cudaMemcpyDeviceToDevice, s));
        for (int64_t k = 0; k + 1 < m; ++k) {
            float* nxt = snap.p + QN * (size_t)(k + 1);
            launch_psm_step(A, snap.p + QN * (size_t)k, nxt, eps.p, s);
            launch_psm_boundary(A, nxt, c->src, (unsigned long long)(tg + k + 1), s);
        }
        for (int64_t k = m - 1; k >= 0; --k) {
            const int64_t t = tg + k;  // step t -> t + 1
            launch_psm_adj_boundary(A, lam0.p, source_shape(c->src, t + 1), grads.p + GRAD_COPIES, s);
            launch_psm_adj_step(A, lam0.p, snap.p + QN * (size_t)k, lam1.p, eps.p, (float)dl[(size_t)t], grads.p,
                                G.p, s);
            lam0.swap(lam1);
        }
        CK(cudaGetLastError());
    }
    launch_psm_grad_x(A, G.p, eps.p, X.p, c->Rd.p, n, dX.p, s);
    CK(cudaGetLastError());
    double gh[GRAD_COPIES + 1];
    CK(cudaMemcpyAsync(gh, grads.p, sizeof(gh), cudaMemcpyDeviceToHost, s));
    if (dL_dX && n > 0) CK(cudaMemcpyAsync(dL_dX, dX.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double d_tau = 0.0;
    for (int k = 0; k < GRAD_COPIES; ++k) d_tau += gh[k];
    if (loss) *loss = L;
    if (dL_dtau) *dL_dtau = d_tau;
    if (dL_damp) *dL_damp = gh[GRAD_COPIES];
    return lbm_dem_status(c);
}

int lbm_dem_relayout(lbmdem_ctx* c) {
    if (!c) return LBMDEM_ERR_INVALID_ARG;
    if (!c->have_packing) return fail(c, LBMDEM_ERR_STATE, "relayout before set_packing");
    if (c->t % 2) return fail(c, LBMDEM_ERR_STATE, "relayout needs an even step count");
    CK(cudaSetDevice(c->p.device));
    if (int r = relayout(c)) return r;
    CK(cudaMemsetAsync(&c->st.p->max_disp_bits, 0, 2 * sizeof(uint32_t), c->stream));
    c->steps_until_check = 0;
    return lbm_dem_status(c);
}

int lbm_dem_status(lbmdem_ctx* c) {
    if (!c) return LBMDEM_ERR_INVALID_ARG;
    CK(cudaMemcpyAsync(c->st_host, c->st.p, sizeof(DevStats), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    int code = map_status(c->st_host->status);
    if (code) c->status_latched = code;
    return code;
}

__global__ void k_particles_out(Dem D, const double* Fh, const double* Th, double* X, double* V,
                                double* W, double* q, double* F, double* T) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D.n) return;
    float4 d = D.dX[i], c = D.dXc[i], v = D.V[i], w = D.W[i], qq = D.q[i];
    X[3 * i] = D.Xref[3 * i] + (double)d.x - (double)c.x;
    X[3 * i + 1] = D.Xref[3 * i + 1] + (double)d.y - (double)c.y;
    X[3 * i + 2] = D.Xref[3 * i + 2] + (double)d.z - (double)c.z;
    V[3 * i] = v.x;
    V[3 * i + 1] = v.y;
    V[3 * i + 2] = v.z;
    W[3 * i] = w.x;
    W[3 * i + 1] = w.y;
    W[3 * i + 2] = w.z;
    q[4 * i] = qq.x;
    q[4 * i + 1] = qq.y;
    q[4 * i + 2] = qq.z;
    q[4 * i + 3] = qq.w;
    for (int a = 0; a < 3; ++a) {
        double f = 0.0, t = 0.0;
        for (int r = 0; r < NREP; ++r) {
            f += Fh[3 * ((size_t)r * D.n + i) + a];
            t += Th[3 * ((size_t)r * D.n + i) + a];
        }
        F[3 * i + a] = f;
        T[3 * i + a] = t;
    }
}

int lbm_dem_read_particles(lbmdem_ctx* c, double* X, double* V, double* Om, double* quat, double* F_hyd,
                           double* T_hyd) {
    if (!c) return LBMDEM_ERR_INVALID_ARG;
    if (!c->have_packing) return fail(c, LBMDEM_ERR_STATE, "no packing");
    if (c->np == 0) return 0;
    CK(cudaSetDevice(c->p.device));
    size_t n = c->np;
    DBuf<double> buf;
    CK(buf.alloc(19 * n));
    double* d = buf.p;
    Dem D = make_dem(c);
    k_particles_out<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(D, c->Fh.p, c->Th.p, d, d + 3 * n,
                                                                      d + 6 * n, d + 9 * n, d + 13 * n,
                                                                      d + 16 * n);
    CK(cudaGetLastError());
    std::vector<double> h(19 * n);
    CK(cudaMemcpyAsync(h.data(), d, sizeof(double) * 19 * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (X) memcpy(X, h.data(), sizeof(double) * 3 * n);
    if (V) memcpy(V, h.data() + 3 * n, sizeof(double) * 3 * n);
    if (Om) memcpy(Om, h.data() + 6 * n, sizeof(double) * 3 * n);
    if (quat) memcpy(quat, h.data() + 9 * n, sizeof(double) * 4 * n);
    if (F_hyd) memcpy(F_hyd, h.data() + 13 * n, sizeof(double) * 3 * n);
    if (T_hyd) memcpy(T_hyd, h.data() + 16 * n, sizeof(double) * 3 * n);
    return lbm_dem_status(c);
}

int lbm_dem_read_fields(lbmdem_ctx* c, double* rho, double* u, uint8_t* solid) {
    if (!c) return LBMDEM_ERR_INVALID_ARG;
    if (!c->have_packing) return fail(c, LBMDEM_ERR_STATE, "no packing");
    if (!c->lbm) return fail(c, LBMDEM_ERR_STATE, "fluid is off");
    CK(cudaSetDevice(c->p.device));
    size_t N = c->N;
    DBuf<double> dr, du;
    DBuf<uint8_t> ds;
    if (rho) CK(dr.alloc(N));
    if (u) CK(du.alloc(3 * N));
    if (solid) CK(ds.alloc(N));
    Lat L = make_lat(c);
    launch_read_fields(L, (c->t & 1) == 1, rho ? dr.p : nullptr, u ? du.p : nullptr, solid ? ds.p : nullptr,
                       c->stream);
    CK(cudaGetLastError());
    if (rho) CK(cudaMemcpyAsync(rho, dr.p, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream));
    if (u) CK(cudaMemcpyAsync(u, du.p, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, c->stream));
    if (solid) CK(cudaMemcpyAsync(solid, ds.p, N, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return lbm_dem_status(c);
}

int lbm_dem_read_plane_means(lbmdem_ctx* c, double* rho, double* jx) {
    if (!c) return LBMDEM_ERR_INVALID_ARG;
    if (!c->have_packing) return fail(c, LBMDEM_ERR_STATE, "no packing");
    if (!c->lbm) return fail(c, LBMDEM_ERR_STATE, "fluid is off");
    CK(cudaSetDevice(c->p.device));
    const int nx = c->p.nx;
    DBuf<double> d;
    CK(d.alloc(3 * (size_t)nx));
    CK(cudaMemsetAsync(d.p, 0, sizeof(double) * 3 * nx, c->stream));
    launch_plane_sums(make_lat(c), (c->t & 1) == 1, d.p, c->stream);
    CK(cudaGetLastError());
    std::vector<double> h(3 * (size_t)nx);
    CK(cudaMemcpyAsync(h.data(), d.p, sizeof(double) * 3 * nx, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int x = 0; x < nx; ++x) {
        double n = h[3 * x + 2];
        if (rho) rho[x] = n > 0 ? c->p.rho_f + h[3 * x] / n : nan("");
        if (jx) jx[x] = n > 0 ? h[3 * x + 1] / n : nan("");
    }
    return lbm_dem_status(c);
}

__global__ void k_probe_out(const double* sums, int64_t n, double rho_f, double* out) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double cnt = sums[2 * k + 1];
    out[k] = cnt > 0 ? rho_f + sums[2 * k] / cnt : nan("");
}

int lbm_dem_read_probe(lbmdem_ctx* c, double* trace, int64_t max_len, int64_t* len) {
    if (!c) return LBMDEM_ERR_INVALID_ARG;
    if (len) *len = c->p.probe_x >= 0 && c->lbm ? c->t : 0;
    if (c->p.probe_x < 0 || !c->lbm || c->t == 0 || !trace || max_len <= 0) return lbm_dem_status(c);
    CK(cudaSetDevice(c->p.device));
    int64_t n = std::min<int64_t>(max_len, c->t);
    DBuf<double> d;
    CK(d.alloc(n));
    k_probe_out<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->probe.p, n, c->p.rho_f, d.p);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(trace, d.p, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return lbm_dem_status(c);
}

__global__ void k_monitors_out(const DevStats* s, double rho_f, double* out) {
    if (threadIdx.x || blockIdx.x) return;
    out[0] = rho_f * s->mon[4] + s->mon[0];
    out[1] = s->mon[1];
    out[2] = s->mon[2];
    out[3] = s->mon[3];
    out[4] = sqrt((double)__uint_as_float(s->max_u_bits));
}

int lbm_dem_read_monitors(lbmdem_ctx* c, double out[6]) {
    if (!c || !out) return LBMDEM_ERR_INVALID_ARG;
    if (!c->lbm) return fail(c, LBMDEM_ERR_STATE, "fluid is off");
    DBuf<double> d;
    CK(d.alloc(6));
    k_monitors_out<<<1, 1, 0, c->stream>>>(c->st.p, c->p.rho_f, d.p);
    CK(cudaMemcpyAsync(out, d.p, sizeof(double) * 5, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    out[5] = (double)c->mon_step;
    return lbm_dem_status(c);
}

int lbm_dem_read_counters(lbmdem_ctx* c, int64_t out[10]) {
    if (!c || !out) return LBMDEM_ERR_INVALID_ARG;
    CK(cudaMemcpyAsync(c->st_host, c->st.p, sizeof(DevStats), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    int64_t fluid = 0;
    if (c->lbm && c->nS) {
        // fluid nodes now: popcount of the compact fluid bits (host reduce of a
        // device array; counters are diagnostics, not part of the step)
        std::vector<uint32_t> fb(c->nSpad / 32);
        CK(cudaMemcpy(fb.data(), c->fbits.p, sizeof(uint32_t) * fb.size(), cudaMemcpyDeviceToHost));
        for (uint32_t w : fb) fluid += __builtin_popcount(w);
    }
    int64_t nb = 0;
    if (c->np) {
        std::vector<int> cnt(c->np);
        CK(cudaMemcpy(cnt.data(), c->nb_cnt.p, sizeof(int) * c->np, cudaMemcpyDeviceToHost));
        for (int v : cnt) nb += v;
    }
    out[0] = (int64_t)c->N;
    out[1] = c->nS;
    out[2] = fluid;
    out[3] = c->nband;
    out[4] = (int64_t)c->nlink_raw;
    out[5] = nb;
    out[6] = c->t;
    out[7] = c->relayouts;
    out[8] = (int64_t)c->st_host->flips_total;
    out[9] = c->launches;
    return 0;
}

int lbm_dem_set_timing(lbmdem_ctx* c, int32_t enable) {
    if (!c) return LBMDEM_ERR_INVALID_ARG;
    if (int r = collect_timing(c)) return r;
    c->timing = enable != 0;
    for (int g = 0; g < NGROUP; ++g) {
        c->tm_ms[g] = 0;
        c->tm_n[g] = 0;
    }
    destroy_graph(c);
    return 0;
}

int lbm_dem_read_timing(lbmdem_ctx* c, double ms[6], int64_t launches[6]) {
    if (!c) return LBMDEM_ERR_INVALID_ARG;
    if (int r = collect_timing(c)) return r;
    for (int g = 0; g < NGROUP; ++g) {
        if (ms) ms[g] = c->tm_ms[g];
        if (launches) launches[g] = c->tm_n[g];
        c->tm_ms[g] = 0;
        c->tm_n[g] = 0;
    }
    return 0;
}

const char* lbm_dem_last_error(const lbmdem_ctx* c) { return c ? c->err.c_str() : "null context"; }

void lbm_dem_destroy(lbmdem_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    destroy_graph(c);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    if (c->st_host) cudaFreeHost(c->st_host);
    if (c->side) cudaStreamSynchronize(c->side);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    cudaSetDevice(c->p.device);
    delete c;  // device buffers are released by their destructors
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Sphere read-out that allocates nothing.
//
// lbm_dem_read_particles stages its output in a device buffer that it
// cudaMallocs and cudaFrees on every call.  Two kinds of caller cannot do
// that: one whose device memory is committed to the lattice state down to
// the last few MB (the cudaMalloc fails), and one that reads the spheres
// while other streams of the process keep the GPU busy and cannot take the
// device-wide synchronisation of cudaFree.  This variant runs the same
// read-out kernel into a fixed file-scope device array and copies from there
// straight into the caller's host arrays.
//
// The array is shared by every call in the process on a given device and
// keeps the last call's contents; nothing in it needs clearing, because the
// kernel writes every value that the call copies out.  Two calls whose work
// overlaps on the GPU (two contexts of one device driven from two host
// threads) race on it.
namespace {
constexpr int NOALLOC_MAX_SPHERES = 65536;  // 19 doubles each: 9.5 MiB
constexpr int NOALLOC_MAX_DEVICES = 64;
__device__ __align__(256) double noalloc_particle_scratch[19 * NOALLOC_MAX_SPHERES];

// The array's address belongs to a CUDA context, not to a device ordinal:
// after cudaDeviceReset (or under another context made current by the
// caller) the device has a new context and the array a new address.  The
// cache is therefore keyed on the device and the unique id of the context
// current at the call (cuCtxGetId, reached through the runtime's driver
// entry points, so no link against the driver library is needed).
struct NoallocSlot {
    unsigned long long ctx_id = 0;
    double* ptr = nullptr;
};
std::mutex noalloc_mutex;
NoallocSlot noalloc_slot[NOALLOC_MAX_DEVICES];
typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long*);
PfnCtxGetCurrent noalloc_get_current = nullptr;
PfnCtxGetId noalloc_get_id = nullptr;

// Unique id of the context current on this thread (0 if none); call with
// noalloc_mutex held.
cudaError_t noalloc_context_id(unsigned long long* id) {
    *id = 0;
    if (!noalloc_get_current || !noalloc_get_id) {
        cudaDriverEntryPointQueryResult q1, q2;
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e != cudaSuccess) return e;
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return e;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return cudaErrorSymbolNotFound;
        noalloc_get_current = (PfnCtxGetCurrent)f1;
        noalloc_get_id = (PfnCtxGetId)f2;
    }
    CUcontext ctx = nullptr;
    if (noalloc_get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaSuccess;
    if (noalloc_get_id(ctx, id) != CUDA_SUCCESS) *id = 0;
    return cudaSuccess;
}

// Device address of the array on device `dev` (which must be current):
// looked up on the first call on the device's current context, and again
// whenever the context changed since.
int noalloc_scratch(lbmdem_ctx* c, int dev, double** out) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return fail(c, LBMDEM_ERR_INVALID_ARG, "read_particles_noalloc: device %d beyond %d", dev,
                    NOALLOC_MAX_DEVICES);
    std::lock_guard<std::mutex> lock(noalloc_mutex);
    unsigned long long id = 0;
    CK(noalloc_context_id(&id));
    NoallocSlot& sl = noalloc_slot[dev];
    if (!sl.ptr || id == 0 || sl.ctx_id != id) {
        double* p = nullptr;
        CK(cudaGetSymbolAddress((void**)&p, noalloc_particle_scratch));
        if (id == 0) CK(noalloc_context_id(&id));  // the lookup created the context
        sl.ptr = p;
        sl.ctx_id = id;
    }
    *out = sl.ptr;
    return 0;
}
}  // namespace

extern "C" int lbm_dem_read_particles_noalloc(lbmdem_ctx* c, double* X, double* V, double* Om, double* quat,
                                              double* F_hyd, double* T_hyd) {
    if (!c) return LBMDEM_ERR_INVALID_ARG;
    if (!c->have_packing) return fail(c, LBMDEM_ERR_STATE, "no packing");
    if (c->np == 0) return 0;
    if (c->np > NOALLOC_MAX_SPHERES)
        return fail(c, LBMDEM_ERR_CAPACITY,
                    "read_particles_noalloc: %d spheres exceed its fixed buffer of %d spheres "
                    "(use lbm_dem_read_particles)",
                    (int)c->np, NOALLOC_MAX_SPHERES);
    CK(cudaSetDevice(c->p.device));
    double* d = nullptr;
    if (int r = noalloc_scratch(c, c->p.device, &d)) return r;
    size_t n = c->np;
    Dem D = make_dem(c);
    k_particles_out<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(D, c->Fh.p, c->Th.p, d, d + 3 * n,
                                                                      d + 6 * n, d + 9 * n, d + 13 * n,
                                                                      d + 16 * n);
    CK(cudaGetLastError());
    double* dst[6] = {X, V, Om, quat, F_hyd, T_hyd};
    const size_t off[6] = {0, 3 * n, 6 * n, 9 * n, 13 * n, 16 * n};
    const size_t len[6] = {3 * n, 3 * n, 3 * n, 4 * n, 3 * n, 3 * n};
    for (int k = 0; k < 6; ++k)
        if (dst[k])
            CK(cudaMemcpyAsync(dst[k], d + off[k], sizeof(double) * len[k], cudaMemcpyDeviceToHost,
                               c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return lbm_dem_status(c);
}
