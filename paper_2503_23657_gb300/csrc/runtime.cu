// Host runtime of libbte: the C ABI declared in include/bte.h.
//
// bte_create builds the sweep plan once (direction ordering by octant, cell
// flags, boundary-face table, per-side normalisers) and uploads it.  bte_solve
// runs the outer source iteration of the paper's solution procedure (Methods,
// steps 1-4): every iteration is one sweep launch (all bands x directions x
// cells) followed by one FP64 update launch (temperature, diffuse inflow,
// eps_T).  Iterations are replayed from a captured CUDA graph, polled every
// few iterations through a device-side convergence flag.  Iteration i reads
// state set i%2 and writes set (i+1)%2, so after n iterations the inputs of
// the last sweep are still available; the final e is regenerated from them by
// one more sweep (outer-iterate checkpointing: T and the diffuse inflow
// determine e).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/bte.h"
#include "bte_internal.cuh"

using namespace bte;

namespace {

constexpr double kFourPi = 4.0 * M_PI;

// An NVTX range around a public entry point (named as the entry point): the
// calls show in Nsight timelines next to their kernels; without a tool
// attached the push and pop cost a function call each.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
thread_local std::string g_create_error;

// Debug mode (environment variable BTE_DEBUG set to anything but 0, read
// once): every device buffer carries kGuardBytes of a fixed pattern after its
// end, and the public entry points check every live buffer's guard after
// they ran (BTE_ECORRUPT names the first overwritten one); plan creation also
// checks its index tables against their extents.
constexpr size_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;
bool debug_mode() {
    static const bool on = [] {
        const char *v = std::getenv("BTE_DEBUG");
        return v != nullptr && v[0] != '\0' && !(v[0] == '0' && v[1] == '\0');
    }();
    return on;
}
struct DevBuf;
std::mutex g_guard_mu;
std::set<const DevBuf *> g_guarded;   // live buffers with a guard (debug mode)

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    bool guarded = false;
    ~DevBuf() { release(); }
    void release() {
        if (guarded) {
            std::lock_guard<std::mutex> lk(g_guard_mu);
            g_guarded.erase(this);
            guarded = false;
        }
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t ensure(size_t n) {
        if (n <= bytes && p) return cudaSuccess;
        release();
        if (n == 0) n = 16;
        const bool dbg = debug_mode();
        cudaError_t e = cudaMalloc(&p, dbg ? n + kGuardBytes : n);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = n;
        if (dbg) {
            e = cudaMemset(static_cast<char *>(p) + n, kGuardByte, kGuardBytes);
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return e;
            std::lock_guard<std::mutex> lk(g_guard_mu);
            g_guarded.insert(this);
            guarded = true;
        }
        return cudaSuccess;
    }
    // debug mode: whether the guard after the buffer still holds its pattern
    bool guard_intact() const {
        if (!guarded || !p) return true;
        unsigned char h[kGuardBytes];
        if (cudaMemcpy(h, static_cast<const char *>(p) + bytes, kGuardBytes, cudaMemcpyDeviceToHost) != cudaSuccess)
            return false;
        for (size_t i = 0; i < kGuardBytes; ++i)
            if (h[i] != kGuardByte) return false;
        return true;
    }
    template <typename T>
    T *as() const { return reinterpret_cast<T *>(p); }
};

// Debug mode: check every live guarded buffer (all plans and batches of the
// process); the number of overwritten guards.
int check_guards() {
    if (!debug_mode()) return 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return -1;
    std::lock_guard<std::mutex> lk(g_guard_mu);
    int bad = 0;
    for (const DevBuf *b : g_guarded) bad += b->guard_intact() ? 0 : 1;
    return bad;
}

struct Status {
    int done;
    int iter;
    int status;
    int pending;   // deferred finalization: the last update's residual is not yet reduced
    double last[3];
};

template <typename real>
struct Workspace {
    bool init = false;
    DevBuf tdev[2], ein[2], T[2];      // forward state sets
    DevBuf thdev[2], mein[2], theta[2];  // adjoint state sets
    DevBuf ein_fixed, part, fsum, e, gpart, phi, coef, invdiag, srck_f, srck_a, qb, cb4pi;
    DevBuf wgt_f, wgt_a, Kinv, scale_f, scale_a, msum, g, grad_out, inv_tt, qcoef, phi64, vws, qshift, q,
        eshift, tfwd_dummy;
    DevBuf wsum;                       // sharded solves: per-cell band-weighted sums [N] (FP64)
    // direction subsets per tile width
    std::map<int, std::pair<std::vector<Subset>, std::vector<Subset>>> subsets;  // tile -> (fwd, adj)
    std::map<int, std::pair<DevBuf *, DevBuf *>> dsub;
    std::vector<std::unique_ptr<DevBuf>> subbufs;
    std::map<int, int> tuned;  // tile request -> chosen tile
    DevBuf wall;  // [6][wall_stride] face index of each wall position (-1: none)
    DevBuf fin_fwd, fin_adj;  // UpdateParams<real> read by the finalize kernel (forward / adjoint)
    DevBuf gradpart;  // gradient reduction block partials
    DevBuf wrap;      // plane-pipeline 3D sweep: last plane of a pass, per CTA
    DevBuf spec[2], mspec[2];  // [B][Fs][D] specular-face inflow (forward / adjoint state sets)
    // extra source of the general kernel's forward sweeps (transient steps:
    // the previous step's e over dt; second-order faces: the deferred
    // correction), and the buffers behind it
    const real *xsrc = nullptr;
    real xscale = real(0);
    DevBuf eprev, del, corr, glpart, ttmp, Tstep;
    // plane-pipeline 3D sweep: skewed copies of the cell records, the source
    // profile and the forward / adjoint sweep sources (both parities)
    // (one set per row axis: [0] rows along y, [1] rows along z)
    DevBuf skc[2], skphi[2], skt[2][2], ska[2][2];
    SkewLayout skew[2]{};
    bool skew_ready[2] = {false, false};
    // graph cache
    cudaGraphExec_t graph = nullptr;
    std::tuple<int, int, double, int> graph_key{-1, -1, 0.0, -1};
    cudaGraphExec_t agraph = nullptr;
    std::tuple<int, int, double, int> agraph_key{-1, -1, 0.0, -1};
    ~Workspace() {
        if (graph) cudaGraphExecDestroy(graph);
        if (agraph) cudaGraphExecDestroy(agraph);
    }
};

}  // namespace

struct bte_plan {
    // problem
    int dim = 0, nx = 1, ny = 1, nz = 1;
    long long N = 0, n_active = 0;
    double h[3] = {1, 1, 1};
    int B = 0, D = 0, R = 0;
    std::vector<double> C, v, tau, tau_scale;
    std::vector<double> s, w;  // internal direction order (sorted by octant)
    std::vector<int> perm;     // internal d -> caller's d
    std::vector<int> groups_d0, groups_cnt, groups_neg;
    int bc_type[6];
    double bc_T[6];
    std::vector<double> phi;  // empty: no source
    std::vector<uint8_t> mask;
    std::vector<int2> cellinfo;
    int F = 0;
    std::vector<int> face_cell, face_side, face_kind;
    int xmode = 0;                    // the current solve: 0 steady step faces, 1 transient step,
                                      // 2 second-order faces (deferred correction)
    double cur_inv_dt = 0.0;          // 1/dt of a transient step (0: steady)
    double forced_T_ref = NAN;        // T_ref kept over the steps of a transient run (NaN: from T_init)
    int solved_order = 1;             // face order of the last solve
    bool want_glen = false;           // the running adjoint forms dJ/dL
    long long spin_limit = kPipeSpinLimit;  // row-pipeline waits (test hook: bte_debug_set_wait_limit)
    double g_L[3] = {0, 0, 0};        // dJ/dL_a of the last bte_adjoint_ex
    std::vector<int> dneg;            // [D] bit a: s_a < 0 (internal order)
    int Fs = 0;                       // specular domain faces
    std::vector<int> sidx;            // [F] specular index of a face (-1: not specular)
    std::vector<int> spec_faces;      // [Fs] face of each specular index
    std::vector<int> mirror;          // [3][D] internal direction with the axis-a component reversed (-1: none)
    double side_norm[6], side_out[6];  // sum over entering / leaving dirs of w |s.n|
    // device, precision independent
    DevBuf d_cell, d_face_cell, d_face_side, d_face_kind, d_perm, d_status, d_counter, d_blockpart, d_hist;
    DevBuf d_sidx, d_mirror, d_dneg;
    int hist_cap = 0;
    Status *h_status = nullptr;  // pinned
    Workspace<float> ws32;
    Workspace<double> ws64;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // per-sweep timing (bte_set_sweep_timing): an event pair around the sweep
    // of every time_every-th iteration of a graph (0 = off)
    int time_every = 0;
    std::vector<cudaEvent_t> tev;
    std::string err;
    // last forward solve
    bool solved = false;
    int solved_precision = -1;
    int solved_iters = 0;
    // sharded solves (bte_shard_*): precision, tile, state set, iterations
    int shard_prec = -1, shard_tile = 0, shard_par = 0, shard_iters = 0;
    int solved_tile = 0;
    int wall_stride = 1;
    std::vector<int> wall_face;
    bool e_current = false;
    cudaStream_t stream = nullptr;  // stream of the last solve (used by the adjoint)
    double T_ref = 300.0;
    std::vector<double> cur_tau, cur_Tw;
    double cur_Q = 0.0;
    int sm_count = 0;

    ~bte_plan() {
        if (h_status) cudaFreeHost(h_status);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        for (cudaEvent_t e : tev) cudaEventDestroy(e);
    }
};

namespace {
// Device state of a batched solve in one precision.
template <typename real>
struct BatchState {
    DevBuf sweep[2], update[2];  // Sweep2DParams<real>[n], UpdateParams<real>[n] per parity
    DevBuf gsweep[2];            // SweepParams<real>[n] per parity (general-kernel classes)
    cudaGraphExec_t graph = nullptr;
    std::vector<int> graph_key;
    std::map<std::vector<int>, std::vector<int>> tuned;  // tile request -> tile per class
    ~BatchState() {
        if (graph) cudaGraphExecDestroy(graph);
    }
};
}  // namespace

// A batch of 2D instances solved together (one graph of batched launches).
struct bte_batch {
    std::vector<bte_plan *> plans;  // borrowed
    int n = 0;
    struct Cls {
        int nrb, begin, count, nx_max, ny_max;
        int general;                // 0: row-pipeline kernel; 1: general kernel (masks, regions)
        int R_max;
    };
    std::vector<Cls> classes;       // instances with the same 32-row block count and kernel
    std::vector<int> inst;          // instance indices, class by class, largest first
    DevBuf d_inst, d_table, d_status, d_done;
    int upd_blocks = 0;
    int *h_done = nullptr;          // pinned
    std::vector<cudaStream_t> side; // one capture stream per class
    std::vector<cudaEvent_t> join;  // one per class
    cudaEvent_t fork = nullptr, ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t tev[2] = {nullptr, nullptr};  // sweep-phase timing (first iteration of a replay)
    bool time_sweeps = false;
    BatchState<float> bs32;
    BatchState<double> bs64;
    std::string err;
    ~bte_batch() {
        if (h_done) cudaFreeHost(h_done);
        for (cudaStream_t s : side) cudaStreamDestroy(s);
        for (cudaEvent_t e : join) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        for (cudaEvent_t e : tev)
            if (e) cudaEventDestroy(e);
    }
};

namespace {

int fail(bte_plan *p, int code, const std::string &msg) {
    if (p)
        p->err = msg;
    else
        g_create_error = msg;
    return code;
}

// Debug mode: after a public entry point ran, BTE_ECORRUPT if any device
// buffer's guard was overwritten (the call's own result otherwise).
int guard_rc(bte_plan *p, int rc) {
    if (!debug_mode()) return rc;
    const int bad = check_guards();
    if (bad < 0) return fail(p, BTE_ECORRUPT, "debug mode: device synchronisation failed during the guard check");
    if (bad > 0)
        return fail(p, BTE_ECORRUPT, "debug mode: " + std::to_string(bad) + " device buffer guard(s) overwritten");
    return rc;
}

#define CK(plan, expr)                                                                              \
    do {                                                                                            \
        cudaError_t _e = (expr);                                                                    \
        if (_e != cudaSuccess) {                                                                    \
            return fail(plan, _e == cudaErrorMemoryAllocation ? BTE_ENOMEM : BTE_ECUDA,             \
                        std::string(#expr) + ": " + cudaGetErrorString(_e));                        \
        }                                                                                           \
    } while (0)

template <typename T>
cudaError_t upload(DevBuf &d, const std::vector<T> &h) {
    cudaError_t e = d.ensure(sizeof(T) * std::max<size_t>(h.size(), 1));
    if (e != cudaSuccess) return e;
    if (h.empty()) return cudaSuccess;
    return cudaMemcpy(d.p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice);
}

bool is_device_ptr(const void *ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

long long cell_index(const bte_plan *p, int i, int j, int k) { return i + (long long)p->nx * (j + (long long)p->ny * k); }

// A sweep tile: kernel kind (0 = general wavefront kernel, 1 = row-block 2D
// kernel with one partial set per warp, 2 = row-block 2D kernel combining its
// warps' per-cell sums through shared-memory slices, 3 = row-pipeline 2D
// kernel with one partial set per direction group and the per-cell source
// staged in shared memory, 4 = the same kernel reading the source ahead from
// global memory), directions per lane/warp (dw) and directions per CTA chunk
// (cw).  Kind 5 is the plane-pipeline 3D kernel (masked grids): one subset
// of dw directions per CTA, and the cw field holds its warps along z.
struct Tile {
    int kind, dw, cw;
};
inline int tile_id(int kind, int dw, int cw) { return kind * 100000 + cw * 100 + dw; }
inline Tile tile_of(int id) { return Tile{id / 100000, id % 100, (id / 100) % 1000}; }
// the bte_solve_opts.tile_kind value of an internal kernel kind
inline int abi_kind(int kind) { return kind == 0 ? 1 : (kind >= 3 ? 3 : 2); }
inline bool is_rowpipe(int kind) { return kind == 3 || kind == 4; }
inline bool is_pipe3(int kind) { return kind == 5; }
// kernels that finalize each iteration in the next sweep's prologue
inline bool defers_finalize(int kind) { return is_rowpipe(kind) || is_pipe3(kind); }
// directions one CTA handles
inline int tile_cta_dirs(const Tile &t) { return is_pipe3(t.kind) ? t.dw : t.cw; }
inline int source_staged_kind(int kind) { return (kind == 4 || kind == 5) ? 0 : 1; }
// plane-pipeline tiles: cw = H + 20 map, map 0 = rows along y, 1 = rows along z
inline int pipe3_h(const Tile &t) { return t.cw % 20; }
inline int pipe3_map(const Tile &t) { return t.cw / 20; }
inline int pipe3_rows(const bte_plan *p, int map) { return map ? p->nz : p->ny; }
inline int pipe3_planes(const bte_plan *p, int map) { return map ? p->ny : p->nz; }

// Directions of one orientation group split into subsets of at most dw.
std::vector<Subset> make_subsets(const bte_plan *p, int dw, bool flip) {
    std::vector<Subset> out;
    const int resolved = (1 << p->dim) - 1;
    for (size_t g = 0; g < p->groups_d0.size(); ++g) {
        for (int o = 0; o < p->groups_cnt[g]; o += dw) {
            Subset s;
            s.d0 = p->groups_d0[g] + o;
            s.cnt = std::min(dw, p->groups_cnt[g] - o);
            s.neg = flip ? (p->groups_neg[g] ^ resolved) : p->groups_neg[g];
            s.pad = 0;
            out.push_back(s);
        }
    }
    return out;
}

int tile_layers(const bte_plan *p) {
    // 1D/2D: one layer; 3D: the fewest register layers that fit 32 warps
    if (p->dim < 3) return 1;
    const int WY = (p->ny + 31) / 32;
    for (int lz : {1, 2, 4, 8})
        if (WY * ((p->nz + lz - 1) / lz) <= 32) return lz;
    return 0;
}

int rowblock_rb(const bte_plan *p) {
    for (int rb : {1, 2, 3, 4, 5})
        if (32 * rb >= p->ny) return rb;
    return 0;
}

// Row-block 2D kernel: unmasked 1D/2D grid, one region, ny <= 160, and the
// CTA's shared memory (reduction ring for `warps` warps, wall values) fits.
// *stage tells whether the per-cell inputs also fit (else they are read
// from global memory).
bool rowblock_ok(const bte_plan *p, int real_bytes, int *stage, int warps = 1, int ring = 0) {
    const int rb = rowblock_rb(p);
    if (p->dim > 2 || rb == 0 || p->n_active != p->N) return false;
    for (long long c = 0; c < p->N; ++c)
        if (p->mask[c] != 1) return false;
    const size_t lim = 200 * 1024;
    *stage = 1;
    return sweep2d_smem(p->nx, p->ny, 1, p->phi.empty() ? 0 : 1, warps, rb, ring, real_bytes) <= lim;
}

// Row-pipeline 2D kernel: unmasked 1D/2D grid with one region, `groups`
// groups of ceil(ny / 32) warps per CTA (at most 16 warps), shared memory fits.
bool rowpipe_ok(const bte_plan *p, int real_bytes, int groups, int dw, int stage = 1) {
    if (p->dim > 2 || p->n_active != p->N) return false;
    const int nrb = (p->ny + 31) / 32;
    if (groups < 1 || groups * nrb > 16) return false;
    for (long long c = 0; c < p->N; ++c)
        if (p->mask[c] != 1) return false;
    return sweep2dp_smem(p->nx, p->ny, p->phi.empty() ? 0 : 1, groups, dw, stage, real_bytes) <= 200 * 1024;
}

// Plane-pipeline 3D kernel: 3D grid (masks and regions allowed), FP32 with
// 2, 4 or 8 directions per lane, FP64 with 2 or 4, ceil(ny / 32) warps along
// y times H along z (at most 16 warps); a grid of
// more than H planes streams in passes, which needs two warps along z and
// nx >= 4 H + 2 (the next pass reads the last plane of the previous one two
// steps ahead, a chunk after it was written).
bool pipe3_ok(const bte_plan *p, int real_bytes, int dw, int H, int map) {
    if (p->dim != 3 || H < 1 || (real_bytes == 8 && dw > 4)) return false;
    if (p->N >= (1LL << 31) - 1) return false;
    const int n1 = pipe3_rows(p, map), n2 = pipe3_planes(p, map);
    const long long skew_entries = 2LL * n2 * (p->nx + n1 - 1) * (((n1 + 31) / 32) * 32) + 32;
    if (skew_entries >= (1LL << 31) - 1) return false;
    const int WY = (n1 + 31) / 32;
    if (WY * H > 16 || H > n2) return false;
    const int M = (n2 + H - 1) / H;
    if (M > 1 && (H < 2 || p->nx < kPipe3Chunk * H + 2)) return false;
    // a lane's virtual columns (passes x nx) stay well inside the range in
    // which the kernel's float reciprocal division by nx is exact
    if ((long long)M * p->nx + 64 >= (1LL << 22)) return false;
    const int variant = (p->Fs > 0 ? 1 : 0) | (p->xmode == 1 ? 2 : 0);
    return sweep3dp_smem(p->R, WY, H, dw, real_bytes, variant) <= 225 * 1024;
}


// Warps along z offered for the plane-pipeline kernel: the most that fit,
// and about half of that (two CTAs per SM).
std::vector<int> pipe3_heights(const bte_plan *p, int real_bytes, int dw, int map) {
    std::vector<int> out;
    const int WY = (pipe3_rows(p, map) + 31) / 32;
    int hmax = 0;
    for (int H = std::min(16 / std::max(WY, 1), pipe3_planes(p, map)); H >= 1; --H)
        if (pipe3_ok(p, real_bytes, dw, H, map)) {
            hmax = H;
            break;
        }
    if (hmax == 0) return out;
    out.push_back(hmax);
    for (int H = (hmax + 1) / 2; H >= 1 && H < hmax; --H)
        if (pipe3_ok(p, real_bytes, dw, H, map)) {
            out.push_back(H);
            break;
        }
    return out;
}

// Candidate tiles for a precision; kind_req 0 = any, 1 = general only,
// 2 = row-block only, 3 = row-pipeline only.
std::vector<int> tile_candidates(const bte_plan *p, int real_bytes, int kind_req = 0, int dw_req = 0,
                                 int cw_req = 0, int staging_req = 0, int wz_req = 0, int axis_req = 0) {
    std::vector<int> out;
    const int lz = tile_layers(p);
    // the plane pipeline carries specular faces and the extra source of
    // transient steps too (3D grids)
    const bool pipe3_only = p->dim == 3 && (p->Fs > 0 || p->xmode == 1) && p->xmode != 2 &&
                            (long long)p->B * p->Fs * p->D < (1LL << 31);   // 32-bit offsets in the kernel
    if (p->Fs > 0 || p->xmode != 0) {
        // specular faces, transient steps, second-order faces: the general
        // kernel's extended variant
        const int mt = sweep_max_threads(kSpecDW, lz, p->dim == 3);
        const int WY = (p->ny + 31) / 32;
        const int WZ = p->dim == 3 && lz ? (p->nz + lz - 1) / lz : 1;
        if (lz != 0 && (kind_req == 0 || kind_req == 1) && (!dw_req || dw_req == kSpecDW) && mt > 0 &&
            WY * WZ * 32 <= mt)
            out.push_back(tile_id(0, kSpecDW, kSpecDW));
        if (!pipe3_only) return out;
    }
    if (lz != 0 && (kind_req == 0 || kind_req == 1) && !pipe3_only) {
        const bool z = p->dim == 3;
        const int WY = (p->ny + 31) / 32;
        const int WZ = z ? (p->nz + lz - 1) / lz : 1;
        for (int dw : {4, 8, 16}) {
            const int mt = sweep_max_threads(dw, lz, z);
            if (mt > 0 && WY * WZ * 32 <= mt && (!dw_req || dw == dw_req)) out.push_back(tile_id(0, dw, dw));
        }
    }
    int stage = 0;
    int gmax = 0;
    for (int c : p->groups_cnt) gmax = std::max(gmax, c);
    if ((kind_req == 0 || kind_req == 3) && !pipe3_only) {
        for (int stage : {1, 0}) {
            if ((staging_req == 1 && !stage) || (staging_req == 2 && stage)) continue;
            for (int dw : {1, 2, 4, 8}) {
                if (dw_req && dw != dw_req) continue;
                for (int groups : {1, 2, 4, 8, 16}) {
                    if (groups > 1 && dw * groups > gmax) break;
                    if (cw_req && dw * groups != cw_req) continue;
                    if (!rowpipe_ok(p, real_bytes, groups, dw, stage)) continue;
                    out.push_back(tile_id(stage ? 3 : 4, dw, dw * groups));
                }
            }
        }
    }
    if ((kind_req == 0 || kind_req == 3) && staging_req != 1) {
        for (int dw : {2, 4, 8}) {
            if ((dw_req && dw != dw_req) || (cw_req && dw != cw_req)) continue;
            // rows along y, and along z where that differs (a grid whose z
            // extent fills the 32 lanes better)
            for (int map = 0; map < 2; ++map) {
                if (axis_req ? (map != axis_req - 1) : (map == 1 && p->nz == p->ny)) continue;
                if (wz_req) {
                    if (pipe3_ok(p, real_bytes, dw, wz_req, map)) out.push_back(tile_id(5, dw, wz_req + 20 * map));
                    continue;
                }
                for (int H : pipe3_heights(p, real_bytes, dw, map)) out.push_back(tile_id(5, dw, H + 20 * map));
            }
        }
    }
    if ((kind_req == 0 || kind_req == 2) && !pipe3_only && rowblock_ok(p, real_bytes, &stage)) {
        for (int dw : {1, 2, 4}) {
            if (dw_req && dw != dw_req) continue;
            for (int warps : {1, 2, 4, 8, 16}) {
                if (warps > 1 && dw * warps > gmax) break;
                if (cw_req && dw * warps != cw_req) continue;
                if (!rowblock_ok(p, real_bytes, &stage, warps, 0)) continue;
                out.push_back(tile_id(1, dw, dw * warps));  // cw = directions per CTA chunk
            }
        }
    }
    return out;
}

template <typename real>
Workspace<real> &ws_of(bte_plan *p);
template <>
Workspace<float> &ws_of<float>(bte_plan *p) { return p->ws32; }
template <>
Workspace<double> &ws_of<double>(bte_plan *p) { return p->ws64; }

// Cell partial sets a tile writes (direct row-block tiles: one per warp).
int cell_sets(int tid, int chunks) {
    const Tile tl = tile_of(tid);
    return (tl.kind == 1 || is_rowpipe(tl.kind)) ? chunks * (tl.cw / tl.dw) : chunks;
}

// Skewed per-cell inputs of the plane-pipeline 3D sweep (built once per plan
// and precision; the sweep sources follow every update).
template <typename real>
int ensure_skew(bte_plan *p, Workspace<real> &ws, int map) {
    if (ws.skew_ready[map]) return BTE_OK;
    SkewLayout L{};
    L.nx = p->nx;
    L.ny = p->ny;
    L.a1 = 1 + map;
    L.n1 = pipe3_rows(p, map);
    L.nd = p->nx + L.n1 - 1;
    L.nyp = ((L.n1 + 31) / 32) * 32;
    L.fam = (long long)pipe3_planes(p, map) * L.nd * L.nyp;
    const size_t n = 2 * (size_t)L.fam + 32;  // both families + a zero pad entry
    CK(p, ws.skc[map].ensure(sizeof(int2) * n));
    CK(p, cudaMemset(ws.skc[map].p, 0, sizeof(int2) * n));
    CK(p, ws.skphi[map].ensure(sizeof(real) * n));
    CK(p, cudaMemset(ws.skphi[map].p, 0, sizeof(real) * n));
    for (int i = 0; i < 2; ++i) {
        CK(p, ws.skt[map][i].ensure(sizeof(real) * n));
        CK(p, cudaMemset(ws.skt[map][i].p, 0, sizeof(real) * n));
        CK(p, ws.ska[map][i].ensure(sizeof(real) * n));
        CK(p, cudaMemset(ws.ska[map][i].p, 0, sizeof(real) * n));
    }
    CK(p, launch_skew<int2>(p->N, L, p->d_cell.as<int2>(), ws.skc[map].template as<int2>(), 0));
    CK(p, launch_skew<real>(p->N, L, ws.phi.template as<real>(), ws.skphi[map].template as<real>(), 0));
    for (int i = 0; i < 2; ++i)
        CK(p, launch_skew<real>(p->N, L, ws.tdev[i].template as<real>(), ws.skt[map][i].template as<real>(), 0));
    CK(p, cudaDeviceSynchronize());
    ws.skew[map] = L;
    ws.skew_ready[map] = true;
    return BTE_OK;
}

// skewed copy (row-axis map `map`) of a natural-order sweep source of the workspace
template <typename real>
const real *skewed_source(Workspace<real> &ws, const real *tsrc, int map) {
    for (int i = 0; i < 2; ++i) {
        if (tsrc == ws.tdev[i].template as<real>()) return ws.skt[map][i].template as<real>();
        if (tsrc == ws.thdev[i].template as<real>()) return ws.ska[map][i].template as<real>();
    }
    return nullptr;
}

template <typename real>
int ensure_subsets(bte_plan *p, Workspace<real> &ws, int tid) {
    if (ws.dsub.count(tid)) return BTE_OK;
    if (is_pipe3(tile_of(tid).kind))
        if (int rc = ensure_skew(p, ws, pipe3_map(tile_of(tid)))) return rc;
    const int cw = tile_cta_dirs(tile_of(tid));  // directions per CTA (general kernel: cw == dw)
    auto f = make_subsets(p, cw, false);
    auto a = make_subsets(p, cw, true);
    // partial sets and face sums of this tile; a buffer that moves invalidates
    // the captured graphs (their kernel parameters hold the old address)
    {
        const size_t N = (size_t)p->N, B = p->B, F = std::max(p->F, 1);
        const size_t chunks = f.size();
        const size_t Spad = ((size_t)cell_sets(tid, (int)chunks) + 3) & ~(size_t)3;
        void *part0 = ws.part.p, *fsum0 = ws.fsum.p, *wrap0 = ws.wrap.p;
        CK(p, ws.part.ensure(sizeof(real) * Spad * B * N));
        CK(p, ws.fsum.ensure(sizeof(real) * chunks * B * F));
        const Tile tl = tile_of(tid);
        if (is_pipe3(tl.kind) && (pipe3_planes(p, pipe3_map(tl)) + pipe3_h(tl) - 1) / pipe3_h(tl) > 1) {
            const size_t ld = (size_t)((pipe3_rows(p, pipe3_map(tl)) + 31) / 32) * 32;
            CK(p, ws.wrap.ensure(sizeof(real) * chunks * B * (size_t)p->nx * ld * tl.dw));
        }
        if (ws.part.p != part0 || ws.fsum.p != fsum0 || ws.wrap.p != wrap0) {
            if (ws.graph) cudaGraphExecDestroy(ws.graph);
            if (ws.agraph) cudaGraphExecDestroy(ws.agraph);
            ws.graph = nullptr;
            ws.agraph = nullptr;
        }
    }
    ws.subsets[tid] = {f, a};
    ws.subbufs.emplace_back(new DevBuf());
    DevBuf *bf = ws.subbufs.back().get();
    ws.subbufs.emplace_back(new DevBuf());
    DevBuf *ba = ws.subbufs.back().get();
    CK(p, upload(*bf, f));
    CK(p, upload(*ba, a));
    ws.dsub[tid] = {bf, ba};
    return BTE_OK;
}


// Per-solve tables (depend on tau overrides, wall temperatures, Q_amp, T_ref).
template <typename real>
int upload_tables(bte_plan *p, Workspace<real> &ws) {
    const int B = p->B, D = p->D, R = p->R;
    const std::vector<double> &tau = p->cur_tau;
    std::vector<real> coef((size_t)B * D * 8), invd((size_t)R * B * D), srf((size_t)R * B), sra((size_t)R * B),
        qb(B), cb(B);
    std::vector<double> wf((size_t)R * B), wa((size_t)R * B), Kinv(R), scf(6 * B), sca(6 * B), itt((size_t)R * B),
        qc(B), vws((size_t)B * D * 3), qsh(3, 0.0), esh(B);
    double Csum = 0.0;
    for (int b = 0; b < B; ++b) Csum += p->C[b];
    for (int b = 0; b < B; ++b) {
        for (int d = 0; d < D; ++d) {
            double a[3] = {0, 0, 0};
            for (int ax = 0; ax < p->dim; ++ax) a[ax] = p->v[b] * std::fabs(p->s[3 * d + ax]) / p->h[ax];
            real *cf = &coef[((size_t)b * D + d) * 8];
            cf[0] = (real)a[0];
            cf[1] = (real)a[1];
            cf[2] = (real)a[2];
            cf[3] = (real)p->w[d];
            for (int ax = 0; ax < 3; ++ax) cf[4 + ax] = (ax < p->dim) ? (real)(p->w[d] * std::fabs(p->s[3 * d + ax])) : (real)0;
            cf[7] = 0;
            for (int r = 0; r < R; ++r) {
                const double trb = tau[b] * p->tau_scale[r];
                invd[((size_t)r * B + b) * D + d] = (real)(1.0 / (1.0 / trb + p->cur_inv_dt + a[0] + a[1] + a[2]));
            }
            for (int ax = 0; ax < 3; ++ax) vws[((size_t)b * D + d) * 3 + ax] = p->v[b] * p->w[d] * p->s[3 * d + ax];
        }
        qb[b] = (real)(p->C[b] * p->cur_Q / (kFourPi * Csum));
        cb[b] = (real)(p->C[b] / kFourPi);
        qc[b] = p->C[b] / (kFourPi * Csum);
        esh[b] = p->C[b] * p->T_ref / kFourPi;
        for (int ax = 0; ax < 3; ++ax) {
            double sws = 0.0;
            for (int d = 0; d < D; ++d) sws += p->w[d] * p->s[3 * d + ax];
            qsh[ax] += p->v[b] * esh[b] * sws;
        }
    }
    for (int r = 0; r < R; ++r) {
        double K = 0.0;
        for (int b = 0; b < B; ++b) {
            const double trb = tau[b] * p->tau_scale[r];
            srf[(size_t)r * B + b] = (real)(p->C[b] / (kFourPi * trb));
            sra[(size_t)r * B + b] = (real)(1.0 / trb);
            wf[(size_t)r * B + b] = 1.0 / trb;
            wa[(size_t)r * B + b] = p->C[b] / (kFourPi * trb);
            itt[(size_t)r * B + b] = 1.0 / (trb * tau[b]);
            K += p->C[b] / trb;
        }
        Kinv[r] = 1.0 / K;
    }
    for (int side = 0; side < 6; ++side)
        for (int b = 0; b < B; ++b) {
            const double nrm = p->side_norm[side];
            scf[side * B + b] = nrm > 0 ? 1.0 / nrm : 0.0;
            sca[side * B + b] = nrm > 0 ? p->h[side / 2] / (p->v[b] * nrm) : 0.0;
        }
    // isothermal inflow C_b (T_w - T_ref) / (4 pi)
    std::vector<real> efix((size_t)B * std::max(p->F, 1), (real)0);
    for (int f = 0; f < p->F; ++f)
        if (p->face_kind[f] == 0)
            for (int b = 0; b < B; ++b)
                efix[(size_t)b * p->F + f] = (real)(p->C[b] * (p->cur_Tw[p->face_side[f]] - p->T_ref) / kFourPi);
    CK(p, upload(ws.coef, coef));
    CK(p, upload(ws.invdiag, invd));
    CK(p, upload(ws.srck_f, srf));
    CK(p, upload(ws.srck_a, sra));
    CK(p, upload(ws.qb, qb));
    CK(p, upload(ws.cb4pi, cb));
    CK(p, upload(ws.wgt_f, wf));
    CK(p, upload(ws.wgt_a, wa));
    CK(p, upload(ws.Kinv, Kinv));
    CK(p, upload(ws.scale_f, scf));
    CK(p, upload(ws.scale_a, sca));
    CK(p, upload(ws.inv_tt, itt));
    CK(p, upload(ws.qcoef, qc));
    CK(p, upload(ws.vws, vws));
    CK(p, upload(ws.qshift, qsh));
    CK(p, upload(ws.eshift, esh));
    CK(p, upload(ws.ein_fixed, efix));
    return BTE_OK;
}

template <typename real>
int ensure_workspace(bte_plan *p, Workspace<real> &ws) {
    if (ws.init) return BTE_OK;
    const size_t N = (size_t)p->N, B = p->B, F = std::max(p->F, 1);
    for (int i = 0; i < 2; ++i) {
        CK(p, ws.tdev[i].ensure(sizeof(real) * (N + 16)));
        CK(p, ws.ein[i].ensure(sizeof(real) * B * F));
        CK(p, ws.T[i].ensure(sizeof(double) * N));
    }
    // (16 values of padding: the plane pipeline copies rows of whole subsets,
    // which may reach past the last face's row when a subset is not full)
    if (p->Fs > 0)
        for (int i = 0; i < 2; ++i) CK(p, ws.spec[i].ensure(sizeof(real) * (B * (size_t)p->Fs * p->D + 16)));
    // the partial sets are sized by the tiles in use (ensure_subsets)
    std::vector<real> ph(N + 16, (real)0);
    for (size_t c = 0; c < N && !p->phi.empty(); ++c) ph[c] = (real)p->phi[c];
    CK(p, upload(ws.phi, ph));
    ws.init = true;
    return BTE_OK;
}

// ---------------------------------------------------------------------------
// launches of one iteration
// ---------------------------------------------------------------------------
template <typename real>
SweepParams<real> sweep_params(bte_plan *p, Workspace<real> &ws, int tid, bool adj) {
    SweepParams<real> sp{};
    sp.nx = p->nx;
    sp.ny = p->ny;
    sp.nz = p->nz;
    sp.dim = p->dim;
    sp.B = p->B;
    sp.D = p->D;
    sp.F = std::max(p->F, 1);
    sp.R = p->R;
    const int lz = tile_layers(p);
    sp.WY = (p->ny + 31) / 32;
    sp.WZ = (p->dim == 3) ? (p->nz + lz - 1) / lz : 1;
    sp.N = p->N;
    sp.cell = p->d_cell.as<int2>();
    sp.part = ws.part.template as<real>();
    sp.fsum = ws.fsum.template as<real>();
    sp.coef = ws.coef.template as<real>();
    sp.invdiag = ws.invdiag.template as<real>();
    sp.srck = adj ? ws.srck_a.template as<real>() : ws.srck_f.template as<real>();
    sp.qb = ws.qb.template as<real>();
    sp.phi = p->phi.empty() ? nullptr : ws.phi.template as<real>();
    sp.cb4pi = ws.cb4pi.template as<real>();
    auto pr = ws.dsub.at(tid);
    sp.sub = (adj ? pr.second : pr.first)->template as<Subset>();
    sp.S = (int)ws.subsets.at(tid).first.size();
    sp.Spad = (sp.S + 3) & ~3;
    sp.done = p->d_status.as<int>();
    // stage the band's boundary values in shared memory when they fit next to
    // the exchange buffers (<= 200 KB of the 227 KB per CTA)
    const size_t ein_bytes = sizeof(real) * (size_t)sp.F;
    const size_t xchg = sizeof(real) * (size_t)sp.WY * sp.WZ * (2 * lz * 16 + (p->dim == 3 ? 2 * 32 * 16 : 0));
    sp.ein_smem = (ein_bytes + xchg <= 200 * 1024) ? 1 : 0;
    if (p->Fs > 0) {
        sp.sidx = p->d_sidx.as<int>();
        sp.mirror = p->d_mirror.as<int>();
        sp.Fs = p->Fs;
    }
    return sp;
}

// An update runs 128-cell vector blocks when the cell count is a multiple
// of 4 (both forms give the same values).  A one-plan update takes them only
// when they are at least two per SM (a small grid fills the GPU better with
// the scalar 32-cell blocks); batched instances share one launch, so theirs
// always do.
inline bool upd_vec_batch(const bte_plan *p) { return p->N % 4 == 0; }
inline bool upd_vec(const bte_plan *p) {
    return upd_vec_batch(p) && p->N >= 2LL * std::max(p->sm_count, 1) * 128;
}

// Convergence bookkeeping of the plan's solve (forward: with eps history).
FinalizeParams fin_params(bte_plan *p, double tol, bool adj) {
    FinalizeParams f{};
    Status *st = p->d_status.as<Status>();
    f.blockpart = p->d_blockpart.as<double>();
    f.nblocks = update_cell_block_count(p->N, upd_vec(p));  // the update's cell blocks
    f.n_active = p->n_active;
    f.tol = tol;
    f.done = &st->done;
    f.iter = &st->iter;
    f.status = &st->status;
    f.pending = &st->pending;
    f.last = st->last;
    f.eps_hist = adj ? nullptr : p->d_hist.as<double>();
    f.max_hist = p->hist_cap;
    f.batch_done = nullptr;
    return f;
}

template <typename real>
UpdateParams<real> update_params(bte_plan *p, Workspace<real> &ws, int tid, bool adj, double tol) {
    UpdateParams<real> u{};
    u.N = p->N;
    u.B = p->B;
    u.Sf = (int)ws.subsets.at(tid).first.size();
    u.S = cell_sets(tid, u.Sf);
    u.Spad = (u.S + 3) & ~3;
    u.F = p->F;
    u.R = p->R;
    u.adjoint = adj ? 1 : 0;
    u.T_ref = p->T_ref;
    u.cell = p->d_cell.as<int2>();
    auto pr = ws.dsub.at(tid);
    u.sub = (adj ? pr.second : pr.first)->template as<Subset>();
    u.part = ws.part.template as<real>();
    u.fsum = ws.fsum.template as<real>();
    u.g = ws.g.template as<double>();
    u.wgt = adj ? ws.wgt_a.template as<double>() : ws.wgt_f.template as<double>();
    // the same weights in the sweep precision: C_b/(4 pi tau_rb) is the
    // forward source factor, 1/tau_rb the adjoint one
    u.wgtr = adj ? ws.srck_f.template as<real>() : ws.srck_a.template as<real>();
    u.vec = upd_vec(p) ? 1 : 0;
    u.Kinv = ws.Kinv.template as<double>();
    u.face_cell = p->d_face_cell.as<int>();
    u.face_side = p->d_face_side.as<int>();
    u.face_kind = p->d_face_kind.as<int>();
    u.ein_fixed = ws.ein_fixed.template as<real>();
    u.side_scale = adj ? ws.scale_a.template as<double>() : ws.scale_f.template as<double>();
    u.blockpart = p->d_blockpart.as<double>();
    u.counter = p->d_counter.as<unsigned int>();
    Status *st = p->d_status.as<Status>();
    u.done = &st->done;
    u.iter = &st->iter;
    u.status = &st->status;
    u.last = st->last;
    u.eps_hist = p->d_hist.as<double>();
    u.max_hist = p->hist_cap;
    u.tol = tol;
    u.n_active = p->n_active;
    // row-pipeline tiles finalize each iteration in the next sweep's prologue
    u.defer = defers_finalize(tile_of(tid).kind) ? 1 : 0;
    if (is_pipe3(tile_of(tid).kind)) u.skew = ws.skew[pipe3_map(tile_of(tid))];
    u.fin = fin_params(p, tol, adj);
    return u;
}

template <typename real>
Sweep2DParams<real> sweep2d_params(bte_plan *p, Workspace<real> &ws, int tid, bool adj) {
    const Tile tl = tile_of(tid);
    Sweep2DParams<real> sp{};
    sp.nx = p->nx;
    sp.ny = p->ny;
    sp.B = p->B;
    sp.D = p->D;
    sp.F = std::max(p->F, 1);
    sp.warps_per_cta = tl.cw / tl.dw;
    sp.part = ws.part.template as<real>();
    sp.fsum = ws.fsum.template as<real>();
    sp.coef = ws.coef.template as<real>();
    sp.invdiag = ws.invdiag.template as<real>();
    sp.srck = adj ? ws.srck_a.template as<real>() : ws.srck_f.template as<real>();
    sp.qb = ws.qb.template as<real>();
    sp.phi = p->phi.empty() ? nullptr : ws.phi.template as<real>();
    auto pr = ws.dsub.at(tid);
    sp.sub = (adj ? pr.second : pr.first)->template as<Subset>();
    sp.S = (int)ws.subsets.at(tid).first.size();
    sp.ring = tl.kind == 2 ? 1 : 0;
    sp.adj = adj ? 1 : 0;
    sp.Spad = (cell_sets(tid, sp.S) + 3) & ~3;
    sp.wall_face = ws.wall.template as<int>();
    sp.wall_stride = p->wall_stride;
    sp.done = p->d_status.as<int>();
    sp.status = &p->d_status.as<Status>()->status;
    sp.spin_limit = p->spin_limit;
    int stage = 0;
    rowblock_ok(p, (int)sizeof(real), &stage, sp.warps_per_cta, sp.ring);
    sp.stage = stage;
    if (is_rowpipe(tl.kind)) {
        sp.groups = tl.cw / tl.dw;
        sp.warps_per_cta = sp.groups * ((p->ny + 31) / 32);
        sp.stage = tl.kind == 3 ? 1 : 0;
    }
    return sp;
}

template <typename real>
Sweep3DParams<real> sweep3d_params(bte_plan *p, Workspace<real> &ws, int tid, bool adj) {
    const Tile tl = tile_of(tid);
    Sweep3DParams<real> sp{};
    sp.nx = p->nx;
    sp.ny = p->ny;
    sp.nz = p->nz;
    sp.B = p->B;
    sp.D = p->D;
    sp.F = std::max(p->F, 1);
    sp.S = (int)ws.subsets.at(tid).first.size();
    sp.R = p->R;
    sp.Spad = (cell_sets(tid, sp.S) + 3) & ~3;
    const int map = pipe3_map(tl);
    sp.lane_axis = 1 + map;
    sp.WY = (pipe3_rows(p, map) + 31) / 32;
    sp.H = pipe3_h(tl);
    sp.N = p->N;
    sp.skew = ws.skew[map];
    sp.cell = ws.skc[map].template as<int2>();
    sp.phi = p->phi.empty() ? nullptr : ws.skphi[map].template as<real>();
    sp.part = ws.part.template as<real>();
    sp.fsum = ws.fsum.template as<real>();
    sp.e = ws.e.template as<real>();
    sp.wrap = ws.wrap.template as<real>();
    auto pr = ws.dsub.at(tid);
    sp.sub = (adj ? pr.second : pr.first)->template as<Subset>();
    sp.coef = ws.coef.template as<real>();
    sp.invdiag = ws.invdiag.template as<real>();
    sp.srck = adj ? ws.srck_a.template as<real>() : ws.srck_f.template as<real>();
    sp.qb = ws.qb.template as<real>();
    sp.done = p->d_status.as<int>();
    sp.adj = adj ? 1 : 0;
    if (p->Fs > 0) {
        sp.Fs = p->Fs;
        sp.sidx = p->d_sidx.as<int>();
        sp.mirror = p->d_mirror.as<int>();
    }
    return sp;
}

// One sweep (all bands x directions x cells) with the given tile.
template <typename real>
cudaError_t launch_tile_sweep(bte_plan *p, Workspace<real> &ws, int tid, bool adj, const real *tsrc,
                              const real *ein, bool store_e, bool use_done, cudaStream_t stream,
                              const FinalizeParams *fin = nullptr, const real *spec_in = nullptr,
                              real *spec_out = nullptr, int b0 = 0, int nb = 0) {
    const Tile tl = tile_of(tid);
    if (is_pipe3(tl.kind)) {
        Sweep3DParams<real> sp = sweep3d_params(p, ws, tid, adj);
        sp.b0 = b0;
        sp.nb = nb;
        sp.tsrc = skewed_source(ws, tsrc, pipe3_map(tl));
        if (!sp.tsrc) return cudaErrorInvalidValue;
        sp.ein = ein;
        sp.store_e = store_e ? 1 : 0;
        sp.spec_in = spec_in;
        sp.spec_out = spec_out;
        if (p->Fs > 0 && !spec_in) return cudaErrorInvalidValue;
        if (!adj && p->xmode == 1) {
            sp.xsrc = ws.xsrc;
            sp.xscale = ws.xscale;
        }
        if (!use_done) sp.done = nullptr;
        if (use_done && fin) sp.fin = *fin;  // finalize the previous iteration
        return launch_sweep3dp<real>(sp, tl.dw, stream);
    }
    if (tl.kind >= 1) {
        Sweep2DParams<real> sp = sweep2d_params(p, ws, tid, adj);
        sp.b0 = b0;
        sp.nb = nb;
        sp.tsrc = tsrc;
        sp.ein = ein;
        sp.store_e = store_e ? 1 : 0;
        sp.e = ws.e.template as<real>();
        if (!use_done) sp.done = nullptr;
        if (use_done && fin && is_rowpipe(tl.kind)) sp.fin = *fin;  // finalize the previous iteration
        if (is_rowpipe(tl.kind)) return launch_sweep2dp<real>(sp, tl.dw, stream);
        return launch_sweep2d<real>(sp, tl.dw, rowblock_rb(p), adj, stream);
    }
    SweepParams<real> sp = sweep_params(p, ws, tid, adj);
    sp.b0 = b0;
    sp.nb = nb;
    sp.tsrc = tsrc;
    sp.ein = ein;
    sp.store_e = store_e ? 1 : 0;
    sp.e = ws.e.template as<real>();
    sp.spec_in = spec_in;
    sp.spec_out = spec_out;
    if (!adj && p->xmode != 0) {
        sp.xsrc = ws.xsrc;
        sp.xscale = ws.xscale;
    }
    if (!use_done) sp.done = nullptr;
    return launch_sweep<real>(sp, tl.dw, tile_layers(p), p->dim == 3, adj, stream);
}

// a timing event: inside a stream capture it must become an event-record
// node of the graph (a plain record only marks a fork/join point there)
inline cudaError_t record_timing_event(cudaEvent_t ev, cudaStream_t stream) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) return e;
    if (cap == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(ev, stream, cudaEventRecordExternal);
    return cudaEventRecord(ev, stream);
}

// Second-order faces: reconstruction increments of the previous iterate
// (ws.e), the next sweep's inflow values rebuilt from them, and its
// deferred-correction source (ws.corr).
template <typename real>
cudaError_t enqueue_order2(bte_plan *p, Workspace<real> &ws, int parity, bool use_done, cudaStream_t stream) {
    Order2Params<real> o{};
    o.N = p->N;
    o.NBD = (long long)p->N * p->B * p->D;
    o.nx = p->nx;
    o.ny = p->ny;
    o.dim = p->dim;
    o.B = p->B;
    o.D = p->D;
    o.F = std::max(p->F, 1);
    o.Fs = p->Fs;
    o.cell = p->d_cell.as<int2>();
    o.e = ws.e.template as<real>();
    o.coef = ws.coef.template as<real>();
    o.dneg = p->d_dneg.as<int>();
    o.face_kind = p->d_face_kind.as<int>();
    o.sidx = p->Fs ? p->d_sidx.as<int>() : nullptr;
    o.mirror = p->Fs ? p->d_mirror.as<int>() : nullptr;
    o.ein_fixed = ws.ein_fixed.template as<real>();
    o.side_scale = ws.scale_f.template as<double>();
    o.del = ws.del.template as<real>();
    o.corr = ws.corr.template as<real>();
    o.ein_out = ws.ein[parity].template as<real>();
    o.spec_out = p->Fs ? ws.spec[parity].template as<real>() : nullptr;
    o.done = use_done ? p->d_status.as<int>() : nullptr;
    return launch_order2<real>(o, stream);
}

template <typename real>
cudaError_t enqueue_forward(bte_plan *p, Workspace<real> &ws, int tid, int parity, double tol, bool store_e,
                            bool replay, cudaStream_t stream, cudaEvent_t ta = nullptr, cudaEvent_t tb = nullptr) {
    if (p->xmode == 2 && !replay) {
        const cudaError_t e2 = enqueue_order2(p, ws, parity, true, stream);
        if (e2 != cudaSuccess) return e2;
        store_e = true;   // the next iteration reconstructs from this one
    }
    cudaError_t e = ta ? record_timing_event(ta, stream) : cudaSuccess;
    const FinalizeParams fin = fin_params(p, tol, false);
    if (e == cudaSuccess)
        e = launch_tile_sweep(p, ws, tid, false, ws.tdev[parity].template as<real>(), ws.ein[parity].template as<real>(),
                              store_e, !replay, stream, &fin, ws.spec[parity].template as<real>(),
                              ws.spec[parity ^ 1].template as<real>());
    if (e == cudaSuccess && tb) e = record_timing_event(tb, stream);
    if (e != cudaSuccess || replay) return e;
    UpdateParams<real> u = update_params(p, ws, tid, false, tol);
    u.x_in = ws.T[parity].template as<double>();
    u.x_out = ws.T[parity ^ 1].template as<double>();
    u.xdev_out = ws.tdev[parity ^ 1].template as<real>();
    if (is_pipe3(tile_of(tid).kind)) u.xskew_out = ws.skt[pipe3_map(tile_of(tid))][parity ^ 1].template as<real>();
    u.ein_out = ws.ein[parity ^ 1].template as<real>();
    return launch_update<real>(u, stream);
}

template <typename real>
int begin_state(bte_plan *p, const bte_solve_opts *o, Workspace<real> &ws, cudaStream_t stream) {
    const long long N = p->N;
    std::vector<double> T0(N);
    if (o->T_init) {
        if (is_device_ptr(o->T_init)) {
            CK(p, cudaMemcpy(T0.data(), o->T_init, sizeof(double) * N, cudaMemcpyDeviceToHost));
        } else {
            std::memcpy(T0.data(), o->T_init, sizeof(double) * N);
        }
    } else {
        std::fill(T0.begin(), T0.end(), o->T_init_uniform);
    }
    double sum = 0.0;
    for (long long c = 0; c < N; ++c) {
        if (!p->mask[c]) {
            T0[c] = 0.0;
            continue;
        }
        if (!(T0[c] > 0.0) || !std::isfinite(T0[c])) return fail(p, BTE_EINVAL, "T_init must be finite and > 0 in solid cells");
        sum += T0[c];
    }
    p->T_ref = std::isnan(p->forced_T_ref) ? sum / (double)p->n_active : p->forced_T_ref;
    std::vector<real> td(N);
    for (long long c = 0; c < N; ++c) td[c] = p->mask[c] ? (real)(T0[c] - p->T_ref) : (real)0;
    const int B = p->B, F = std::max(p->F, 1);
    std::vector<real> e0((size_t)B * F, (real)0);
    std::vector<double> ein0;
    if (o->ein_init && p->F > 0) {
        ein0.resize((size_t)B * p->F);
        if (is_device_ptr(o->ein_init)) {
            CK(p, cudaMemcpy(ein0.data(), o->ein_init, sizeof(double) * ein0.size(), cudaMemcpyDeviceToHost));
        } else {
            std::memcpy(ein0.data(), o->ein_init, sizeof(double) * ein0.size());
        }
        for (double v : ein0)
            if (!std::isfinite(v)) return fail(p, BTE_EINVAL, "ein_init must be finite");
    }
    for (int f = 0; f < p->F; ++f) {
        const long long c = p->face_cell[f];
        const int side = p->face_side[f];
        for (int b = 0; b < B; ++b) {
            double val;
            if (p->face_kind[f] == 0)
                val = p->C[b] * (p->cur_Tw[side] - p->T_ref) / kFourPi;
            else if (!ein0.empty())  // resume: the inflow of the state the caller saved
                val = ein0[(size_t)b * p->F + f] - p->C[b] * p->T_ref / kFourPi;
            else  // diffuse reflection of the initial equilibrium e0(T_init)
                val = p->C[b] * (T0[c] - p->T_ref) / kFourPi * p->side_out[side] / p->side_norm[side];
            e0[(size_t)b * F + f] = (real)val;
        }
    }
    CK(p, cudaMemcpyAsync(ws.T[0].p, T0.data(), sizeof(double) * N, cudaMemcpyHostToDevice, stream));
    CK(p, cudaMemcpyAsync(ws.tdev[0].p, td.data(), sizeof(real) * N, cudaMemcpyHostToDevice, stream));
    for (int map = 0; map < 2; ++map)
        if (ws.skew_ready[map])
            CK(p, launch_skew<real>(N, ws.skew[map], ws.tdev[0].template as<real>(), ws.skt[map][0].template as<real>(),
                                    stream));
    CK(p, cudaMemcpyAsync(ws.ein[0].p, e0.data(), sizeof(real) * e0.size(), cudaMemcpyHostToDevice, stream));
    std::vector<real> s0;
    if (p->Fs > 0) {
        // the initial e = e0(T_init) is isotropic: every mirror direction carries it
        s0.resize((size_t)B * p->Fs * p->D);
        for (int b = 0; b < B; ++b)
            for (int k = 0; k < p->Fs; ++k) {
                const long long c = p->face_cell[p->spec_faces[k]];
                const real v = (real)(p->C[b] * (T0[c] - p->T_ref) / kFourPi);
                std::fill(s0.begin() + ((size_t)b * p->Fs + k) * p->D, s0.begin() + ((size_t)b * p->Fs + k + 1) * p->D, v);
            }
        CK(p, cudaMemcpyAsync(ws.spec[0].p, s0.data(), sizeof(real) * s0.size(), cudaMemcpyHostToDevice, stream));
    }
    CK(p, cudaMemsetAsync(p->d_status.p, 0, sizeof(Status), stream));
    CK(p, cudaMemsetAsync(p->d_counter.p, 0, sizeof(unsigned int), stream));
    CK(p, cudaStreamSynchronize(stream));
    return BTE_OK;
}

// Pick the fastest candidate tile by timing whole iterations (sweep +
// update) on the current state; the caller re-initialises the state after.
template <typename real>
int autotune(bte_plan *p, Workspace<real> &ws, const std::vector<int> &cand, cudaStream_t stream) {
    if (cand.empty()) return 0;
    if (cand.size() == 1) return cand[0];
    float best = 1e30f;
    int best_tid = cand[0];
    for (int tid : cand) {
        if (ensure_subsets(p, ws, tid) != BTE_OK) return 0;
        float tmin = 1e30f;
        for (int rep = 0; rep < 6; ++rep) {
            cudaEventRecord(p->ev0, stream);
            if (enqueue_forward(p, ws, tid, rep & 1, 0.0, false, false, stream) != cudaSuccess) {
                cudaGetLastError();
                tmin = 1e30f;
                break;
            }
            cudaEventRecord(p->ev1, stream);
            cudaEventSynchronize(p->ev1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, p->ev0, p->ev1);
            if (rep >= 2) tmin = std::min(tmin, ms);
        }
        if (std::getenv("BTE_TUNE_VERBOSE"))
            std::fprintf(stderr, "bte tune: kind %d dw %d cw %d: %.4f ms/iteration\n", abi_kind(tile_of(tid).kind),
                         tile_of(tid).dw, tile_of(tid).cw, tmin);
        if (tmin < best) {
            best = tmin;
            best_tid = tid;
        }
    }
    return best_tid;
}

// event pair i brackets the sweep of iteration i of a graph replay
cudaError_t ensure_timing_events(bte_plan *p, int pairs) {
    while ((int)p->tev.size() < 2 * pairs) {
        cudaEvent_t e;
        cudaError_t ce = cudaEventCreate(&e);
        if (ce != cudaSuccess) return ce;
        p->tev.push_back(e);
    }
    return cudaSuccess;
}

bool timed_iter(const bte_plan *p, int i) { return p->time_every > 0 && i % p->time_every == 0; }
cudaEvent_t tev_a(bte_plan *p, int i) { return timed_iter(p, i) ? p->tev[2 * (i / p->time_every)] : nullptr; }
cudaEvent_t tev_b(bte_plan *p, int i) { return timed_iter(p, i) ? p->tev[2 * (i / p->time_every) + 1] : nullptr; }

// after the stream reached the last of k iterations (global indices base ..
// base + k - 1): add the durations of their timed sweeps (ms) and count them,
// leaving out the iterations at or past `ran` (the iterations the solve has
// finished): a replay's iterations after convergence return at once and
// would pull the mean sweep time down; cudaSuccess only if every counted
// pair was recorded
cudaError_t sum_timing_events(bte_plan *p, int k, int base, int ran, double *ms, long long *n) {
    for (int i = 0; i < k; ++i) {
        if (!timed_iter(p, i) || base + i >= ran) continue;
        float t = 0.f;
        const cudaError_t e = cudaEventElapsedTime(&t, tev_a(p, i), tev_b(p, i));
        if (e != cudaSuccess) return e;
        *ms += t;
        *n += 1;
    }
    return cudaSuccess;
}

template <typename real>
int solve_t(bte_plan *p, const bte_solve_opts *o, double *T_out, double *q_out, void *e_out, bte_stats *st) {
    cudaStream_t stream = (cudaStream_t)o->stream;
    Workspace<real> &ws = ws_of<real>(p);
    int rc = ensure_workspace(p, ws);
    if (rc) return rc;
    // per-solve parameters
    p->cur_tau = p->tau;
    if (o->tau) {
        for (int b = 0; b < p->B; ++b)
            if (!(o->tau[b] > 0.0) || !std::isfinite(o->tau[b])) return fail(p, BTE_EINVAL, "tau override must be > 0");
        p->cur_tau.assign(o->tau, o->tau + p->B);
    }
    p->cur_Tw.assign(p->bc_T, p->bc_T + 6);
    if (o->T_wall) p->cur_Tw.assign(o->T_wall, o->T_wall + 6);
    p->cur_Q = o->Q_amp;
    if ((rc = begin_state(p, o, ws, stream))) return rc;
    if ((rc = upload_tables(p, ws))) return rc;
    // tile: the caller's restriction, then the autotuned choice (cached)
    if (o->tile_kind < 0 || o->tile_kind > 3) return fail(p, BTE_EINVAL, "tile_kind must be 0, 1, 2 or 3");
    if (o->source_staging < 0 || o->source_staging > 2) return fail(p, BTE_EINVAL, "source_staging must be 0, 1 or 2");
    if (o->warps_z < 0 || o->warps_z > 16) return fail(p, BTE_EINVAL, "warps_z must be in 0..16");
    if (o->lane_axis < 0 || o->lane_axis > 2) return fail(p, BTE_EINVAL, "lane_axis must be 0, 1 or 2");
    std::vector<int> cand = tile_candidates(p, (int)sizeof(real), o->tile_kind, o->dirs_per_lane, o->dirs_per_cta,
                                            o->source_staging, o->warps_z, o->lane_axis);
    if (cand.empty()) return fail(p, BTE_EINVAL, "no sweep tile supports this grid / tile request");
    const int tkey =
        (((((p->xmode * 3 + o->lane_axis) * 20 + o->warps_z) * 10 + o->source_staging) * 10 + o->tile_kind) * 100 +
         o->dirs_per_lane) *
            1000 +
        o->dirs_per_cta;
    int tid;
    if (ws.tuned.count(tkey)) {
        tid = ws.tuned[tkey];
    } else {
        tid = autotune(p, ws, cand, stream);
        if (!tid) return fail(p, BTE_ECUDA, "tile autotuning failed");
        ws.tuned[tkey] = tid;
    }
    const int dw = tid;
    if ((rc = ensure_subsets(p, ws, dw))) return rc;
    // e of the final iterate is always regenerated on the device (outputs and
    // the adjoint read it)
    const size_t NBD = (size_t)p->N * p->B * p->D;
    {
        // zeros where no sweep writes (void cells): the e of a transient step
        // is the next step's extra source, read for every cell
        const void *e0 = ws.e.p;
        CK(p, ws.e.ensure(sizeof(real) * NBD));
        if (ws.e.p != e0) CK(p, cudaMemsetAsync(ws.e.p, 0, sizeof(real) * NBD, stream));
    }
    if (p->xmode == 2) {
        CK(p, ws.del.ensure(sizeof(real) * 3 * NBD));
        CK(p, ws.corr.ensure(sizeof(real) * NBD));
        CK(p, cudaMemsetAsync(ws.corr.p, 0, sizeof(real) * NBD, stream));
        ws.xsrc = ws.corr.template as<real>();
        ws.xscale = real(1);
    }
    const double tol = o->tol;
    // one launch outside any capture sets the kernel's shared-memory attribute
    CK(p, enqueue_forward(p, ws, dw, 0, tol, false, true, stream));
    // re-initialise after autotuning / the warm launch touched the work buffers
    if ((rc = begin_state(p, o, ws, stream))) return rc;
    if (p->xmode == 2) {
        // the previous iterate of the first iteration: the equilibrium at T_init
        CK(p, launch_equilibrium<real>(p->N, p->B, p->D, p->d_cell.as<int2>(), ws.tdev[0].template as<real>(),
                                       ws.cb4pi.template as<real>(), ws.e.template as<real>(), stream));
    }
    int poll = o->poll_every > 0 ? o->poll_every : 32;
    poll = std::max(2, poll + (poll & 1));
    const bool store_every = o->store_e_every_iter != 0;
    if (p->time_every) CK(p, ensure_timing_events(p, poll));
    // graph of `poll` iterations (even, so every replay starts at parity 0)
    auto key = std::make_tuple(dw, poll, tol + 1e3 * p->cur_inv_dt,
                               (store_every ? 1 : 0) | (p->xmode << 1) | (p->time_every << 3));
    // the finalize kernel that closes every replay / eager chunk (a no-op
    // unless the tile defers finalization)
    {
        const UpdateParams<real> uf = update_params(p, ws, dw, false, tol);
        CK(p, ws.fin_fwd.ensure(sizeof(UpdateParams<real>)));
        CK(p, cudaMemcpy(ws.fin_fwd.p, &uf, sizeof(UpdateParams<real>), cudaMemcpyHostToDevice));
    }
    const UpdateParams<real> *fin_fwd = ws.fin_fwd.template as<UpdateParams<real>>();
    if (!ws.graph || ws.graph_key != key) {
        if (ws.graph) {
            cudaGraphExecDestroy(ws.graph);
            ws.graph = nullptr;
        }
        cudaStream_t cs;
        CK(p, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g;
        cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        for (int i = 0; i < poll && ce == cudaSuccess; ++i)
            ce = enqueue_forward(p, ws, dw, i & 1, tol, store_every, false, cs, tev_a(p, i), tev_b(p, i));
        if (ce == cudaSuccess) ce = launch_finalize<real>(fin_fwd, 1, cs);
        cudaError_t ce2 = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (ce != cudaSuccess) return fail(p, BTE_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        if (ce2 != cudaSuccess) return fail(p, BTE_ECUDA, std::string("graph capture end: ") + cudaGetErrorString(ce2));
        ce = cudaGraphInstantiate(&ws.graph, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) {
            ws.graph = nullptr;
            return fail(p, BTE_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
        }
        ws.graph_key = key;
    }
    const int max_iter = o->max_iter;
    int enq = 0;
    long long launches = 0;
    double sweep_ms = 0.0;
    long long n_timed = 0;
    CK(p, cudaEventRecord(p->ev0, stream));
    while (enq < max_iter) {
        const int k = std::min(poll, max_iter - enq);
        if (k == poll) {
            CK(p, cudaGraphLaunch(ws.graph, stream));
        } else {
            for (int i = 0; i < k; ++i)
                CK(p, enqueue_forward(p, ws, dw, (enq + i) & 1, tol, store_every, false, stream, tev_a(p, i), tev_b(p, i)));
            CK(p, launch_finalize<real>(fin_fwd, 1, stream));
        }
        enq += k;
        launches += 2LL * k + 1;
        CK(p, cudaMemcpyAsync(p->h_status, p->d_status.p, sizeof(Status), cudaMemcpyDeviceToHost, stream));
        CK(p, cudaStreamSynchronize(stream));
        if (p->time_every) CK(p, sum_timing_events(p, k, enq - k, p->h_status->iter, &sweep_ms, &n_timed));
        if (p->h_status->done || p->h_status->status) break;
    }
    CK(p, cudaEventRecord(p->ev1, stream));
    CK(p, cudaEventSynchronize(p->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p->ev0, p->ev1);
    const int n = p->h_status->iter;
    const int sflag = p->h_status->status;
    const bool bad = sflag != 0;
    const bool converged = tol > 0.0 && p->h_status->done && !bad;
    if (sflag == 2) return fail(p, BTE_ETIMEOUT, "a bounded device wait (bulk copy) expired");
    // eps_q (solution procedure, step 4; reported, not used to stop): the
    // change of |q| over one more iteration from the returned state, from the
    // e of iteration n + 1 (swept from the kept inputs of iteration n; not
    // with specular faces, whose inflow arrays that sweep would overwrite)
    double eps_q = NAN;
    const bool want_eps_q = q_out && st && n > 0 && p->Fs == 0 && p->xmode == 0;
    std::vector<double> q_next;
    if (want_eps_q) {
        CK(p, ws.q.ensure(sizeof(double) * 3 * p->N));
        CK(p, enqueue_forward(p, ws, dw, n & 1, tol, true, true, stream));
        CK(p, launch_flux<real>(p->N, p->B, p->D, p->d_cell.as<int2>(), ws.e.template as<real>(), ws.vws.template as<double>(),
                                ws.qshift.template as<double>(), ws.q.template as<double>(), stream));
        launches += 2;
        q_next.resize(3 * (size_t)p->N);
        CK(p, cudaMemcpyAsync(q_next.data(), ws.q.p, sizeof(double) * 3 * p->N, cudaMemcpyDeviceToHost, stream));
    }
    // regenerate e^n from the inputs of the last iteration
    if (n > 0) CK(p, enqueue_forward(p, ws, dw, (n - 1) & 1, tol, true, true, stream));
    if (n > 0) launches += 1;
    p->e_current = n > 0;
    const int par = n & 1;
    CK(p, cudaMemcpyAsync(T_out, ws.T[par].p, sizeof(double) * p->N, cudaMemcpyDefault, stream));
    if (q_out && n > 0) {
        CK(p, ws.q.ensure(sizeof(double) * 3 * p->N));
        CK(p, launch_flux<real>(p->N, p->B, p->D, p->d_cell.as<int2>(), ws.e.template as<real>(), ws.vws.template as<double>(),
                                ws.qshift.template as<double>(), ws.q.template as<double>(), stream));
        launches += 1;
        CK(p, cudaMemcpyAsync(q_out, ws.q.p, sizeof(double) * 3 * p->N, cudaMemcpyDefault, stream));
        if (want_eps_q) {
            std::vector<double> q_now(3 * (size_t)p->N);
            CK(p, cudaMemcpyAsync(q_now.data(), ws.q.p, sizeof(double) * 3 * p->N, cudaMemcpyDeviceToHost, stream));
            CK(p, cudaStreamSynchronize(stream));
            double ss = 0.0, qmax = 0.0;
            for (long long c = 0; c < p->N; ++c) {
                if (!p->mask[c]) continue;
                const double *a = &q_now[3 * c], *b2 = &q_next[3 * c];
                const double m0 = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
                const double m1 = std::sqrt(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]);
                ss += (m0 - m1) * (m0 - m1);
                qmax = std::max(qmax, m1);
            }
            eps_q = qmax > 0.0 ? std::sqrt(ss / (double)p->n_active) / qmax : 0.0;
        }
    }
    if (e_out && n > 0) {
        const size_t ne = (size_t)p->N * p->B * p->D;
        if (is_device_ptr(e_out)) {
            CK(p, launch_permute_e<real>(p->N, p->B, p->D, p->d_cell.as<int2>(), ws.e.template as<real>(), p->d_perm.as<int>(),
                                         ws.eshift.template as<double>(), (real *)e_out, stream));
            launches += 1;
        } else {
            CK(p, cudaMemcpyAsync(e_out, ws.e.p, sizeof(real) * ne, cudaMemcpyDeviceToHost, stream));
            CK(p, cudaStreamSynchronize(stream));
            real *eo = (real *)e_out;
            std::vector<real> tmp(p->D);
            for (size_t cb = 0; cb < (size_t)p->N * p->B; ++cb) {
                const int b = (int)(cb % p->B);
                const double sh = p->mask[cb / p->B] ? p->C[b] * p->T_ref / kFourPi : 0.0;
                for (int d = 0; d < p->D; ++d)
                    tmp[p->perm[d]] = p->mask[cb / p->B] ? (real)((double)eo[cb * p->D + d] + sh) : (real)0;
                std::memcpy(eo + cb * p->D, tmp.data(), sizeof(real) * p->D);
            }
        }
    }
    CK(p, cudaStreamSynchronize(stream));
    p->solved = true;
    p->stream = stream;
    p->solved_order = p->xmode == 2 ? 2 : 1;
    p->solved_precision = (sizeof(real) == 4) ? BTE_FP32 : BTE_FP64;
    p->solved_iters = n;
    p->solved_tile = tid;
    if (st) {
        st->iterations = n;
        st->converged = converged ? 1 : 0;
        st->eps_T = p->h_status->last[0];
        st->T_max = p->h_status->last[1];
        st->seconds = ms * 1e-3;
        st->updates_per_s = st->seconds > 0 ? (double)n * p->n_active * p->B * p->D / st->seconds : 0.0;
        st->dirs_per_lane = tile_of(tid).dw;
        st->tile_kind = abi_kind(tile_of(tid).kind);
        st->dirs_per_cta = tile_cta_dirs(tile_of(tid));
        st->kernel_launches = launches;
        st->sweep_seconds = sweep_ms * 1e-3;
        st->sweep_launches = n_timed;
        st->source_staged = source_staged_kind(tile_of(tid).kind);
        st->warps_z = is_pipe3(tile_of(tid).kind) ? pipe3_h(tile_of(tid)) : 0;
        st->lane_axis = is_pipe3(tile_of(tid).kind) ? 1 + pipe3_map(tile_of(tid)) : 0;
        st->eps_q = eps_q;
    }
    if (bad) return fail(p, BTE_ENUMERIC, "NaN or Inf in the temperature update");
    if (tol > 0.0 && !converged) return fail(p, BTE_ENOTCONVERGED, "max_iter reached before eps_T < tol");
    return BTE_OK;
}

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------
template <typename real>
cudaError_t enqueue_adjoint(bte_plan *p, Workspace<real> &ws, int dw, int parity, double tol, bool final_pass,
                            cudaStream_t stream, cudaEvent_t ta = nullptr, cudaEvent_t tb = nullptr) {
    if (!final_pass) {
        cudaError_t e = ta ? record_timing_event(ta, stream) : cudaSuccess;
        const FinalizeParams fin = fin_params(p, tol, true);
        if (e == cudaSuccess)
            e = launch_tile_sweep(p, ws, dw, true, ws.thdev[parity].template as<real>(), ws.mein[parity].template as<real>(),
                                  false, true, stream, &fin, ws.mspec[parity].template as<real>(),
                                  ws.mspec[parity ^ 1].template as<real>());
        if (e == cudaSuccess && tb) e = record_timing_event(tb, stream);
        if (e != cudaSuccess) return e;
        UpdateParams<real> u = update_params(p, ws, dw, true, tol);
        u.eps_hist = nullptr;
        u.x_in = ws.theta[parity].template as<double>();
        u.x_out = ws.theta[parity ^ 1].template as<double>();
        u.xdev_out = ws.thdev[parity ^ 1].template as<real>();
        if (is_pipe3(tile_of(dw).kind)) u.xskew_out = ws.ska[pipe3_map(tile_of(dw))][parity ^ 1].template as<real>();
        u.ein_out = ws.mein[parity ^ 1].template as<real>();
        return launch_update<real>(u, stream);
    }
    cudaError_t e;
    if (is_pipe3(tile_of(dw).kind)) {
        // the final pass on the plane pipeline: the transposed sweep (partial
        // sets and face sums), then the same sweep in its gradient form (the
        // dJ/dtau partials, into gpart), both from Theta^n
        const int map = pipe3_map(tile_of(dw));
        Sweep3DParams<real> a3 = sweep3d_params(p, ws, dw, true);
        a3.tsrc = skewed_source(ws, ws.thdev[parity].template as<real>(), map);
        if (!a3.tsrc) return cudaErrorInvalidValue;
        a3.ein = ws.mein[parity].template as<real>();
        a3.done = nullptr;
        a3.iso_fsum = 1;   // the wall-temperature gradients read them
        if (p->Fs > 0) {
            a3.spec_in = ws.mspec[parity].template as<real>();
            a3.spec_out = ws.mspec[parity ^ 1].template as<real>();
        }
        e = launch_sweep3dp<real>(a3, tile_of(dw).dw, stream);
        if (e != cudaSuccess) return e;
        Sweep3DParams<real> g3 = sweep3d_params(p, ws, dw, true);
        g3.tsrc = skewed_source(ws, ws.thdev[parity].template as<real>(), map);
        if (!g3.tsrc) return cudaErrorInvalidValue;
        g3.ein = ws.mein[parity].template as<real>();
        g3.done = nullptr;
        g3.grad = 1;
        g3.part = ws.gpart.template as<real>();
        g3.tfwd = ws.skt[map][p->solved_iters & 1].template as<real>();   // T^n of the solve
        g3.cb4pi = ws.cb4pi.template as<real>();
        if (p->Fs > 0) g3.spec_in = ws.mspec[parity].template as<real>();
        e = launch_sweep3dp<real>(g3, tile_of(dw).dw, stream);
    } else {
        SweepParams<real> sp = sweep_params(p, ws, dw, true);
        sp.tsrc = ws.thdev[parity].template as<real>();
        sp.ein = ws.mein[parity].template as<real>();
        sp.e = ws.e.template as<real>();
        sp.gpart = ws.gpart.template as<real>();
        sp.read_e = final_pass ? 1 : 0;
        sp.tfwd = ws.tdev[p->solved_iters & 1].template as<real>();
        sp.spec_in = ws.mspec[parity].template as<real>();
        sp.spec_out = ws.mspec[parity ^ 1].template as<real>();
        if (final_pass && p->want_glen) {
            // cell-size partials against the inflow the final forward e was made from
            const int fpar = (p->solved_iters - 1) & 1;
            sp.glpart = ws.glpart.template as<real>();
            sp.ein_fwd = ws.ein[fpar].template as<real>();
            sp.spec_fwd = p->Fs ? ws.spec[fpar].template as<real>() : nullptr;
        }
        if (final_pass) sp.done = nullptr;
        e = launch_sweep<real>(sp, tile_of(dw).dw, tile_layers(p), p->dim == 3, true, stream);
    }
    if (e != cudaSuccess) return e;
    UpdateParams<real> u = update_params(p, ws, dw, true, tol);
    u.eps_hist = nullptr;  // the history belongs to the forward solve
    u.x_in = ws.theta[parity].template as<double>();
    u.x_out = ws.theta[parity ^ 1].template as<double>();
    u.xdev_out = ws.thdev[parity ^ 1].template as<real>();
    u.ein_out = ws.mein[parity ^ 1].template as<real>();
    if (final_pass) {
        u.ignore_done = 1;
        u.defer = 0;
        u.fsum_total = ws.msum.template as<double>();
    }
    return launch_update<real>(u, stream);
}

template <typename real>
int adjoint_t(bte_plan *p, const double *dJ_dT, double tol, int max_iter, double *g_tau, double *g_Tw, double *g_Q,
              double *g_L, bte_stats *st) {
    cudaStream_t stream = p->stream;
    Workspace<real> &ws = ws_of<real>(p);
    const int dw = p->solved_tile;
    // the final gradient pass reads e and runs on a general tile (the
    // extended variant when it also forms the cell-size partials)
    // the final pass runs on the solve's own tile where that is the plane
    // pipeline (its gradient form), else on a general tile
    const bool pipe_grad = is_pipe3(tile_of(dw).kind) && !g_L;
    int gtile = dw;
    if (!pipe_grad) {
        std::vector<int> gen = tile_candidates(p, (int)sizeof(real), 1, g_L ? kSpecDW : 0);
        if (gen.empty()) return fail(p, BTE_EINVAL, "no general sweep tile for the gradient pass");
        gtile = gen[0];
        if (int rc2 = ensure_subsets(p, ws, gtile)) return rc2;
    }
    const long long N = p->N;
    const int B = p->B, F = std::max(p->F, 1);
    const size_t S = ws.subsets.at(gtile).first.size();  // the gradient pass: one set per chunk
    const size_t Spad = ((size_t)cell_sets(gtile, (int)S) + 3) & ~(size_t)3;
    for (int i = 0; i < 2; ++i) {
        CK(p, ws.thdev[i].ensure(sizeof(real) * (N + 16)));
        CK(p, ws.mein[i].ensure(sizeof(real) * (size_t)B * F));
        CK(p, ws.theta[i].ensure(sizeof(double) * N));
    }
    if (p->Fs > 0) {
        for (int i = 0; i < 2; ++i) CK(p, ws.mspec[i].ensure(sizeof(real) * ((size_t)B * p->Fs * p->D + 16)));
    }
    CK(p, ws.gpart.ensure(sizeof(real) * Spad * B * N));
    if (g_L) CK(p, ws.glpart.ensure(sizeof(real) * 3 * Spad * B * N));
    CK(p, ws.msum.ensure(sizeof(double) * (size_t)B * F));
    CK(p, ws.g.ensure(sizeof(double) * N));
    CK(p, ws.grad_out.ensure(sizeof(double) * (B + 10)));
    std::vector<double> g(N);
    if (is_device_ptr(dJ_dT)) {
        CK(p, cudaMemcpyAsync(g.data(), dJ_dT, sizeof(double) * N, cudaMemcpyDeviceToHost, stream));
        CK(p, cudaStreamSynchronize(stream));
    } else {
        std::memcpy(g.data(), dJ_dT, sizeof(double) * N);
    }
    // Theta^0 = g / K (mu^0 = 0), M^0 = 0
    std::vector<double> K(p->R);
    for (int r = 0; r < p->R; ++r) {
        double k = 0.0;
        for (int b = 0; b < B; ++b) k += p->C[b] / (p->cur_tau[b] * p->tau_scale[r]);
        K[r] = k;
    }
    std::vector<double> th(N, 0.0);
    std::vector<real> thr(N, (real)0);
    for (long long c = 0; c < N; ++c) {
        if (!p->mask[c]) {
            g[c] = 0.0;
            continue;
        }
        if (!std::isfinite(g[c])) return fail(p, BTE_EINVAL, "dJ_dT must be finite");
        th[c] = g[c] / K[p->mask[c] - 1];
        thr[c] = (real)th[c];
    }
    CK(p, cudaMemcpyAsync(ws.g.p, g.data(), sizeof(double) * N, cudaMemcpyHostToDevice, stream));
    CK(p, cudaMemcpyAsync(ws.theta[0].p, th.data(), sizeof(double) * N, cudaMemcpyHostToDevice, stream));
    CK(p, cudaMemcpyAsync(ws.thdev[0].p, thr.data(), sizeof(real) * N, cudaMemcpyHostToDevice, stream));
    for (int map = 0; map < 2; ++map)
        if (ws.skew_ready[map])
            CK(p, launch_skew<real>(N, ws.skew[map], ws.thdev[0].template as<real>(), ws.ska[map][0].template as<real>(),
                                    stream));
    CK(p, cudaMemsetAsync(ws.mein[0].p, 0, sizeof(real) * (size_t)B * F, stream));
    if (p->Fs > 0) CK(p, cudaMemsetAsync(ws.mspec[0].p, 0, sizeof(real) * (size_t)B * p->Fs * p->D, stream));
    CK(p, cudaMemsetAsync(p->d_status.p, 0, sizeof(Status), stream));
    CK(p, cudaMemsetAsync(p->d_counter.p, 0, sizeof(unsigned int), stream));
    if (!p->e_current) {
        // regenerate the forward e^n from the stored state of the last solve
        CK(p, enqueue_forward(p, ws, dw, (p->solved_iters - 1) & 1, 0.0, true, true, stream));
        p->e_current = true;
    }
    CK(p, enqueue_adjoint(p, ws, dw, 0, tol, false, stream));   // attribute set outside capture
    CK(p, cudaMemsetAsync(p->d_status.p, 0, sizeof(Status), stream));
    CK(p, cudaMemsetAsync(p->d_counter.p, 0, sizeof(unsigned int), stream));
    const int poll = 32;
    if (p->time_every) CK(p, ensure_timing_events(p, poll));
    {
        const UpdateParams<real> uf = update_params(p, ws, dw, true, tol);
        CK(p, ws.fin_adj.ensure(sizeof(UpdateParams<real>)));
        CK(p, cudaMemcpy(ws.fin_adj.p, &uf, sizeof(UpdateParams<real>), cudaMemcpyHostToDevice));
    }
    const UpdateParams<real> *fin_adj = ws.fin_adj.template as<UpdateParams<real>>();
    auto key = std::make_tuple(dw, poll, tol, p->time_every << 1);
    if (!ws.agraph || ws.agraph_key != key) {
        if (ws.agraph) {
            cudaGraphExecDestroy(ws.agraph);
            ws.agraph = nullptr;
        }
        cudaStream_t cs;
        CK(p, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t gr;
        cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        for (int i = 0; i < poll && ce == cudaSuccess; ++i)
            ce = enqueue_adjoint(p, ws, dw, i & 1, tol, false, cs, tev_a(p, i), tev_b(p, i));
        if (ce == cudaSuccess) ce = launch_finalize<real>(fin_adj, 1, cs);
        cudaError_t ce2 = cudaStreamEndCapture(cs, &gr);
        cudaStreamDestroy(cs);
        if (ce != cudaSuccess || ce2 != cudaSuccess)
            return fail(p, BTE_ECUDA, std::string("adjoint graph capture: ") + cudaGetErrorString(ce != cudaSuccess ? ce : ce2));
        ce = cudaGraphInstantiate(&ws.agraph, gr, 0);
        cudaGraphDestroy(gr);
        if (ce != cudaSuccess) {
            ws.agraph = nullptr;
            return fail(p, BTE_ECUDA, std::string("adjoint graph instantiate: ") + cudaGetErrorString(ce));
        }
        ws.agraph_key = key;
    }
    int enq = 0;
    long long launches = p->e_current ? 0 : 1;
    double sweep_ms = 0.0;
    long long n_timed = 0;
    CK(p, cudaEventRecord(p->ev0, stream));
    while (enq < max_iter) {
        const int k = std::min(poll, max_iter - enq);
        launches += 2LL * k + 1;
        if (k == poll) {
            CK(p, cudaGraphLaunch(ws.agraph, stream));
        } else {
            for (int i = 0; i < k; ++i)
                CK(p, enqueue_adjoint(p, ws, dw, (enq + i) & 1, tol, false, stream, tev_a(p, i), tev_b(p, i)));
            CK(p, launch_finalize<real>(fin_adj, 1, stream));
        }
        enq += k;
        CK(p, cudaMemcpyAsync(p->h_status, p->d_status.p, sizeof(Status), cudaMemcpyDeviceToHost, stream));
        CK(p, cudaStreamSynchronize(stream));
        if (p->time_every) CK(p, sum_timing_events(p, k, enq - k, p->h_status->iter, &sweep_ms, &n_timed));
        if (p->h_status->done || p->h_status->status) break;
    }
    const int n = p->h_status->iter;
    if (p->h_status->status == 2) return fail(p, BTE_ETIMEOUT, "a bounded device wait (bulk copy) expired");
    const bool bad = p->h_status->status != 0;
    const bool converged = tol > 0.0 && p->h_status->done && !bad;
    // final pass: one more transposed sweep from Theta^n that also forms the
    // gradient partials against the forward state, then the face sums
    CK(p, enqueue_adjoint(p, ws, gtile, n & 1, tol, true, stream));
    GradParams<real> gp{};
    gp.N = N;
    gp.B = B;
    gp.S = cell_sets(gtile, (int)S);
    gp.Spad = (int)Spad;
    gp.F = p->F;
    gp.cell = p->d_cell.as<int2>();
    gp.apart = ws.part.template as<real>();
    gp.gpart = ws.gpart.template as<real>();
    if (!p->phi.empty()) {
        CK(p, upload(ws.phi64, p->phi));
        gp.phi = ws.phi64.template as<double>();
    }
    gp.inv_tt = ws.inv_tt.template as<double>();
    gp.qcoef = ws.qcoef.template as<double>();
    std::vector<double> cb(B);
    for (int b = 0; b < B; ++b) cb[b] = p->C[b] / kFourPi;
    CK(p, upload(ws.tfwd_dummy, cb));
    gp.cb4pi = ws.tfwd_dummy.template as<double>();
    gp.face_side = p->d_face_side.as<int>();
    gp.face_kind = p->d_face_kind.as<int>();
    gp.msum = ws.msum.template as<double>();
    gp.glpart = g_L ? ws.glpart.template as<real>() : nullptr;
    const int nblk = (int)((N + 255) / 256) + (p->F + 255) / 256;
    CK(p, ws.gradpart.ensure(sizeof(double) * (size_t)nblk * (B + 10)));
    gp.blockpart = ws.gradpart.template as<double>();
    gp.counter = p->d_counter.as<unsigned int>();
    gp.out = ws.grad_out.template as<double>();
    CK(p, launch_grad<real>(gp, stream));
    std::vector<double> out(B + 10);
    CK(p, cudaMemcpyAsync(out.data(), ws.grad_out.p, sizeof(double) * (B + 10), cudaMemcpyDeviceToHost, stream));
    CK(p, cudaEventRecord(p->ev1, stream));
    CK(p, cudaEventSynchronize(p->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p->ev0, p->ev1);
    if (g_tau) std::memcpy(g_tau, out.data(), sizeof(double) * B);
    if (g_Tw) {
        for (int f = 0; f < 6; ++f) g_Tw[f] = (f / 2 < p->dim && p->bc_type[f] == BTE_BC_ISOTHERMAL) ? out[B + f] : 0.0;
    }
    if (g_Q) *g_Q = out[B + 6];
    if (g_L) {
        // dJ/dL_a = (1/L_a) sum mu a^a (e - e_in): a^a = v |s_a| / h_a, h_a = L_a / n_a
        const int nn[3] = {p->nx, p->ny, p->nz};
        for (int a = 0; a < 3; ++a) g_L[a] = a < p->dim ? out[B + 7 + a] / (p->h[a] * nn[a]) : 0.0;
    }
    if (st) {
        st->eps_q = NAN;
        st->iterations = n;
        st->converged = converged;
        st->eps_T = p->h_status->last[0];
        st->T_max = p->h_status->last[1];
        st->seconds = ms * 1e-3;
        st->updates_per_s = st->seconds > 0 ? (double)(n + 1) * p->n_active * p->B * p->D / st->seconds : 0.0;
        st->dirs_per_lane = tile_of(dw).dw;
        st->tile_kind = abi_kind(tile_of(dw).kind);
        st->dirs_per_cta = tile_cta_dirs(tile_of(dw));
        st->kernel_launches = launches + 3;  // final sweep + update + gradient reduction
        st->sweep_seconds = sweep_ms * 1e-3;
        st->sweep_launches = n_timed;
        st->source_staged = source_staged_kind(tile_of(dw).kind);
        st->warps_z = is_pipe3(tile_of(dw).kind) ? pipe3_h(tile_of(dw)) : 0;
        st->lane_axis = is_pipe3(tile_of(dw).kind) ? 1 + pipe3_map(tile_of(dw)) : 0;
    }
    if (bad) return fail(p, BTE_ENUMERIC, "NaN or Inf in the adjoint update");
    if (tol > 0.0 && !converged) return fail(p, BTE_ENOTCONVERGED, "adjoint: max_iter reached before tol");
    return BTE_OK;
}

// Transient: n_steps implicit-Euler steps of length dt, every one a solve of
// the steady machinery with 1/dt on the diagonal (upload_tables) and the
// previous step's e over dt as the extra source of the sweep (the plane
// pipeline's extra-source variant on 3D grids, else the general kernel's
// extended variant); T_ref stays that of the initial state over the run.
template <typename real>
int transient_t(bte_plan *p, const bte_solve_opts *o, double dt, int n_steps, double *T_out, double *T_hist,
                bte_stats *st) {
    Workspace<real> &ws = ws_of<real>(p);
    cudaStream_t stream = (cudaStream_t)o->stream;
    int rc = ensure_workspace(p, ws);
    if (rc) return rc;
    const long long N = p->N;
    const size_t NBD = (size_t)N * p->B * p->D;
    std::vector<double> T0(N);
    if (o->T_init) {
        if (is_device_ptr(o->T_init)) {
            CK(p, cudaMemcpy(T0.data(), o->T_init, sizeof(double) * N, cudaMemcpyDeviceToHost));
        } else {
            std::memcpy(T0.data(), o->T_init, sizeof(double) * N);
        }
    } else {
        std::fill(T0.begin(), T0.end(), o->T_init_uniform);
    }
    double sum = 0.0;
    std::vector<real> td(N, (real)0);
    for (long long c = 0; c < N; ++c) {
        if (!p->mask[c]) {
            T0[c] = 0.0;
            continue;
        }
        if (!(T0[c] > 0.0) || !std::isfinite(T0[c])) return fail(p, BTE_EINVAL, "T_init must be finite and > 0 in solid cells");
        sum += T0[c];
    }
    const double T_ref = sum / (double)p->n_active;
    for (long long c = 0; c < N; ++c) td[c] = p->mask[c] ? (real)(T0[c] - T_ref) : (real)0;
    CK(p, ws.eprev.ensure(sizeof(real) * (NBD + 16)));   // (padded: the plane pipeline copies whole subsets)
    CK(p, ws.ttmp.ensure(sizeof(real) * (N + 16)));
    CK(p, ws.Tstep.ensure(sizeof(double) * N));
    std::vector<real> cb(p->B);
    for (int b = 0; b < p->B; ++b) cb[b] = (real)(p->C[b] / kFourPi);
    CK(p, upload(ws.cb4pi, cb));
    CK(p, cudaMemcpyAsync(ws.ttmp.p, td.data(), sizeof(real) * N, cudaMemcpyHostToDevice, stream));
    // the initial state is the equilibrium at T_init
    CK(p, launch_equilibrium<real>(N, p->B, p->D, p->d_cell.as<int2>(), ws.ttmp.template as<real>(),
                                   ws.cb4pi.template as<real>(), ws.eprev.template as<real>(), stream));
    CK(p, cudaMemcpyAsync(ws.Tstep.p, T0.data(), sizeof(double) * N, cudaMemcpyHostToDevice, stream));
    CK(p, cudaStreamSynchronize(stream));
    p->forced_T_ref = T_ref;
    p->xmode = 1;
    p->cur_inv_dt = 1.0 / dt;
    ws.xsrc = ws.eprev.template as<real>();
    ws.xscale = (real)(1.0 / dt);
    bte_solve_opts so = *o;
    so.T_init = ws.Tstep.template as<double>();
    int total = 0, all_conv = 1;
    long long launches = 0;
    double secs = 0.0;
    bte_stats sm{};
    for (int m = 0; m < n_steps; ++m) {
        rc = solve_t<real>(p, &so, ws.Tstep.template as<double>(), nullptr, nullptr, &sm);
        if (rc != BTE_OK && rc != BTE_ENOTCONVERGED) return rc;
        if (rc == BTE_ENOTCONVERGED) all_conv = 0;
        total += sm.iterations;
        secs += sm.seconds;
        launches += sm.kernel_launches + 1;
        if (T_hist)
            CK(p, cudaMemcpyAsync(T_hist + (size_t)m * N, ws.Tstep.p, sizeof(double) * N, cudaMemcpyDefault, stream));
        // this step's e (regenerated by the solve) is the next step's previous state
        CK(p, cudaMemcpyAsync(ws.eprev.p, ws.e.p, sizeof(real) * NBD, cudaMemcpyDeviceToDevice, stream));
    }
    CK(p, cudaMemcpyAsync(T_out, ws.Tstep.p, sizeof(double) * N, cudaMemcpyDefault, stream));
    CK(p, cudaStreamSynchronize(stream));
    if (st) {
        *st = sm;
        st->iterations = total;
        st->converged = all_conv;
        st->seconds = secs;
        st->updates_per_s = secs > 0 ? (double)total * p->n_active * p->B * p->D / secs : 0.0;
        st->kernel_launches = launches;
    }
    if (!all_conv) return fail(p, BTE_ENOTCONVERGED, "a time step reached max_iter before eps_T < tol");
    return BTE_OK;
}

template <typename real>
int profile_t(bte_plan *p, int reps, double *ms_per_sweep) {
    Workspace<real> &ws = ws_of<real>(p);
    cudaStream_t stream = p->stream;
    const int par = (p->solved_iters - 1) & 1;
    for (int i = 0; i < 2; ++i) CK(p, enqueue_forward(p, ws, p->solved_tile, par, 0.0, false, true, stream));
    CK(p, cudaEventRecord(p->ev0, stream));
    for (int i = 0; i < reps; ++i) CK(p, enqueue_forward(p, ws, p->solved_tile, par, 0.0, false, true, stream));
    CK(p, cudaEventRecord(p->ev1, stream));
    CK(p, cudaEventSynchronize(p->ev1));
    float ms = 0.f;
    CK(p, cudaEventElapsedTime(&ms, p->ev0, p->ev1));
    *ms_per_sweep = ms / reps;
    return BTE_OK;
}

int build_plan(bte_plan *p, const bte_grid *g, const uint8_t *mask, const bte_bands *bands, const bte_quad *quad,
               const bte_bcs *bcs, const double *q_profile) {
    if (!g || !mask || !bands || !quad || !bcs) return fail(nullptr, BTE_EINVAL, "null argument");
    if (g->dim < 1 || g->dim > 3) return fail(nullptr, BTE_EINVAL, "dim must be 1, 2 or 3");
    for (int a = 0; a < 3; ++a) {
        if (g->n[a] < 1) return fail(nullptr, BTE_EINVAL, "n[a] must be >= 1");
        if (a >= g->dim && g->n[a] != 1) return fail(nullptr, BTE_EINVAL, "n[a] must be 1 for axes >= dim");
        if (!(g->length[a] > 0.0) || !std::isfinite(g->length[a])) return fail(nullptr, BTE_EINVAL, "length must be > 0");
    }
    p->dim = g->dim;
    p->nx = g->n[0];
    p->ny = g->n[1];
    p->nz = g->n[2];
    p->N = (long long)p->nx * p->ny * p->nz;
    if (p->N > (1LL << 31) - 1) return fail(nullptr, BTE_EINVAL, "too many cells");
    for (int a = 0; a < 3; ++a) p->h[a] = g->length[a] / g->n[a];
    if (bands->B < 1 || bands->R < 1 || bands->R > kMaxRegions || !bands->C || !bands->v || !bands->tau || !bands->tau_scale)
        return fail(nullptr, BTE_EINVAL, "bands: need B >= 1, 1 <= R <= 15 and all arrays");
    p->B = bands->B;
    p->R = bands->R;
    p->C.assign(bands->C, bands->C + p->B);
    p->v.assign(bands->v, bands->v + p->B);
    p->tau.assign(bands->tau, bands->tau + p->B);
    p->tau_scale.assign(bands->tau_scale, bands->tau_scale + p->R);
    for (int b = 0; b < p->B; ++b)
        if (!(p->C[b] > 0) || !(p->v[b] > 0) || !(p->tau[b] > 0) || !std::isfinite(p->C[b] * p->v[b] * p->tau[b]))
            return fail(nullptr, BTE_EINVAL, "bands: C, v, tau must be finite and > 0");
    for (int r = 0; r < p->R; ++r)
        if (!(p->tau_scale[r] > 0) || !std::isfinite(p->tau_scale[r]))
            return fail(nullptr, BTE_EINVAL, "bands: tau_scale must be finite and > 0");
    if (quad->D < 1 || !quad->s || !quad->w) return fail(nullptr, BTE_EINVAL, "quad: need D >= 1");
    p->D = quad->D;
    double wsum = 0.0;
    for (int d = 0; d < p->D; ++d) {
        if (!(quad->w[d] > 0) || !std::isfinite(quad->w[d])) return fail(nullptr, BTE_EINVAL, "quad: weights must be > 0");
        wsum += quad->w[d];
        const double n2 = quad->s[3 * d] * quad->s[3 * d] + quad->s[3 * d + 1] * quad->s[3 * d + 1] +
                          quad->s[3 * d + 2] * quad->s[3 * d + 2];
        if (!(std::fabs(n2 - 1.0) < 1e-8)) return fail(nullptr, BTE_EINVAL, "quad: directions must be unit vectors");
    }
    if (std::fabs(wsum - kFourPi) > 1e-10 * kFourPi) return fail(nullptr, BTE_EINVAL, "quad: sum of weights must be 4 pi");
    // internal order: stable sort by orientation key over the resolved axes
    std::vector<int> order(p->D);
    std::vector<int> key(p->D);
    for (int d = 0; d < p->D; ++d) {
        order[d] = d;
        int k = 0;
        for (int a = 0; a < p->dim; ++a) k = k * 2 + (quad->s[3 * d + a] < 0.0 ? 1 : 0);
        key[d] = k;
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return key[x] < key[y]; });
    p->s.resize(3 * p->D);
    p->w.resize(p->D);
    p->perm.resize(p->D);
    for (int d = 0; d < p->D; ++d) {
        for (int a = 0; a < 3; ++a) p->s[3 * d + a] = quad->s[3 * order[d] + a];
        p->w[d] = quad->w[order[d]];
        p->perm[d] = order[d];
    }
    p->dneg.assign(p->D, 0);
    for (int d = 0; d < p->D; ++d)
        for (int a = 0; a < 3; ++a)
            if (p->s[3 * d + a] < 0.0) p->dneg[d] |= 1 << a;
    for (int d = 0; d < p->D;) {
        int e = d;
        while (e < p->D && key[order[e]] == key[order[d]]) ++e;
        int neg = 0;
        for (int a = 0; a < p->dim; ++a)
            if (p->s[3 * d + a] < 0.0) neg |= 1 << a;
        p->groups_d0.push_back(d);
        p->groups_cnt.push_back(e - d);
        p->groups_neg.push_back(neg);
        d = e;
    }
    for (int side = 0; side < 6; ++side) {
        const int a = side / 2;
        const double sg = (side & 1) ? 1.0 : -1.0;
        double nin = 0.0, nout = 0.0;
        for (int d = 0; d < p->D; ++d) {
            const double sn = p->s[3 * d + a] * sg;
            if (sn < 0.0) nin += p->w[d] * std::fabs(sn);
            if (sn > 0.0) nout += p->w[d] * sn;
        }
        p->side_norm[side] = nin;
        p->side_out[side] = nout;
    }
    for (int f = 0; f < 6; ++f) {
        if (bcs->type[f] != BTE_BC_ISOTHERMAL && bcs->type[f] != BTE_BC_DIFFUSE && bcs->type[f] != BTE_BC_SPECULAR)
            return fail(nullptr, BTE_EINVAL, "bcs: unknown face type");
        if (bcs->type[f] == BTE_BC_ISOTHERMAL && f / 2 < p->dim && (!(bcs->T[f] > 0) || !std::isfinite(bcs->T[f])))
            return fail(nullptr, BTE_EINVAL, "bcs: wall temperature must be > 0");
        p->bc_type[f] = bcs->type[f];
        p->bc_T[f] = bcs->T[f];
    }
    // cells and faces
    p->mask.assign(mask, mask + p->N);
    p->cellinfo.resize(p->N);
    bool anchored = false;
    for (int k = 0; k < p->nz; ++k)
        for (int j = 0; j < p->ny; ++j)
            for (int i = 0; i < p->nx; ++i) {
                const long long c = cell_index(p, i, j, k);
                const int r = p->mask[c];
                if (r > p->R) return fail(nullptr, BTE_EINVAL, "mask value exceeds the number of regions");
                int flags = r, base = p->F;
                if (r) {
                    ++p->n_active;
                    const int idx[3] = {i, j, k};
                    for (int side = 0; side < 2 * p->dim; ++side) {
                        const int a = side / 2;
                        int jdx[3] = {i, j, k};
                        jdx[a] += (side & 1) ? 1 : -1;
                        const bool outside = jdx[a] < 0 || jdx[a] >= g->n[a];
                        const bool voidn = !outside && p->mask[cell_index(p, jdx[0], jdx[1], jdx[2])] == 0;
                        (void)idx;
                        if (outside || voidn) {
                            flags |= 1 << (kSideShift + side);
                            p->face_cell.push_back((int)c);
                            p->face_side.push_back(side);
                            const bool iso = outside && p->bc_type[side] == BTE_BC_ISOTHERMAL;
                            const bool spec = outside && p->bc_type[side] == BTE_BC_SPECULAR;
                            p->face_kind.push_back(iso ? 0 : (spec ? 2 : 1));
                            if (iso) flags |= 1 << (kIsoShift + side);
                            if (spec) flags |= 1 << (kSpecShift + side);
                            p->sidx.push_back(spec ? p->Fs : -1);
                            if (spec) {
                                p->spec_faces.push_back(p->F);
                                ++p->Fs;
                            }
                            if (iso) anchored = true;
                            ++p->F;
                        }
                    }
                }
                p->cellinfo[c] = make_int2(base, flags);
            }
    if (p->n_active == 0) return fail(nullptr, BTE_EINVAL, "mask has no solid cell");
    // domain-wall position -> face index (used by the row-block 2D kernel)
    p->wall_stride = std::max((long long)p->ny * p->nz, std::max((long long)p->nx * p->nz, (long long)p->nx * p->ny));
    p->wall_face.assign((size_t)6 * p->wall_stride, -1);
    for (int f = 0; f < p->F; ++f) {
        const long long c = p->face_cell[f];
        const int side = p->face_side[f];
        const int i = (int)(c % p->nx), j = (int)((c / p->nx) % p->ny), k = (int)(c / ((long long)p->nx * p->ny));
        const int a = side / 2;
        const int idx[3] = {i, j, k};
        const bool on_wall = (side & 1) ? idx[a] == g->n[a] - 1 : idx[a] == 0;
        if (!on_wall) continue;
        long long pos = a == 0 ? j + (long long)p->ny * k : (a == 1 ? i + (long long)p->nx * k : i + (long long)p->nx * j);
        p->wall_face[(size_t)side * p->wall_stride + pos] = f;
    }
    if (!anchored) return fail(nullptr, BTE_EINVAL, "no isothermal face touches the solid (temperature undetermined)");
    // mirror directions (internal order) for the specular faces
    p->mirror.assign((size_t)3 * p->D, -1);
    for (int d = 0; d < p->D; ++d)
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < p->D; ++k) {
                double err = 0.0;
                for (int q = 0; q < 3; ++q) err += std::fabs(p->s[3 * k + q] - (q == a ? -p->s[3 * d + q] : p->s[3 * d + q]));
                if (err < 1e-12) {
                    p->mirror[(size_t)a * p->D + d] = k;
                    break;
                }
            }
    for (int f = 0; f < 2 * p->dim; ++f)
        if (p->bc_type[f] == BTE_BC_SPECULAR)
            for (int d = 0; d < p->D; ++d)
                if (p->mirror[(size_t)(f / 2) * p->D + d] < 0)
                    return fail(nullptr, BTE_EINVAL, "quad: a specular face needs the mirror of every direction");
    if (q_profile) {
        p->phi.assign(q_profile, q_profile + p->N);
        for (long long c = 0; c < p->N; ++c)
            if (!std::isfinite(p->phi[c])) return fail(nullptr, BTE_EINVAL, "q_profile must be finite");
    }
    return BTE_OK;
}


// ---------------------------------------------------------------------------
// batched solves (many 2D instances, one graph of batched launches)
// ---------------------------------------------------------------------------
int bfail(bte_batch *bt, int code, const std::string &msg) {
    if (bt)
        bt->err = msg;
    else
        g_create_error = msg;
    return code;
}

#define BCK(bt, expr)                                                                               \
    do {                                                                                            \
        cudaError_t _e = (expr);                                                                    \
        if (_e != cudaSuccess) {                                                                    \
            return bfail(bt, _e == cudaErrorMemoryAllocation ? BTE_ENOMEM : BTE_ECUDA,              \
                         std::string(#expr) + ": " + cudaGetErrorString(_e));                       \
        }                                                                                           \
    } while (0)

template <typename real>
BatchState<real> &bstate_of(bte_batch *bt);
template <>
BatchState<float> &bstate_of<float>(bte_batch *bt) { return bt->bs32; }
template <>
BatchState<double> &bstate_of<double>(bte_batch *bt) { return bt->bs64; }

// Row-pipeline candidates valid for every instance of a class (its largest
// instance needs the most shared memory).
std::vector<int> batch_class_candidates(bte_batch *bt, const bte_batch::Cls &c, int real_bytes, int dw_req,
                                        int cw_req) {
    if (c.general) {
        // the general kernel, 4 or 8 directions per lane
        std::vector<int> out;
        for (int dw : {4, 8}) {
            if (dw_req && dw != dw_req) continue;
            if (sweep_max_threads(dw, 1, false) >= c.nrb * 32) out.push_back(tile_id(0, dw, dw));
        }
        return out;
    }
    std::vector<int> all = tile_candidates(bt->plans[bt->inst[c.begin]], real_bytes, 3, dw_req, cw_req);
    if (dw_req) return all;
    // one direction per warp is never the fastest with this much parallelism
    // and needs the most partial sets per instance
    std::vector<int> out;
    for (int tid : all)
        if (tile_of(tid).dw > 1) out.push_back(tid);
    return out.empty() ? all : out;
}

template <typename real>
Sweep2DBatch<real> batch_launch_desc(bte_batch *bt, BatchState<real> &bs, const bte_batch::Cls &c, int tid,
                                     int parity) {
    const Tile tl = tile_of(tid);
    const bte_plan *p0 = bt->plans[bt->inst[c.begin]];
    Sweep2DBatch<real> d{};
    d.params = bs.sweep[parity].template as<Sweep2DParams<real>>();
    d.inst = bt->d_inst.as<int>() + c.begin;
    d.n_inst = c.count;
    d.chunks = (int)ws_of<real>(bt->plans[bt->inst[c.begin]]).subsets.at(tid).first.size();
    d.B = p0->B;
    d.groups = tl.cw / tl.dw;
    d.nrb = c.nrb;
    d.nx_max = c.nx_max;
    d.ny_max = c.ny_max;
    d.phi = 0;
    d.stage = tl.kind == 3 ? 1 : 0;
    for (int q = 0; q < c.count; ++q)
        if (!bt->plans[bt->inst[c.begin + q]]->phi.empty()) d.phi = 1;
    return d;
}

template <typename real>
SweepBatch<real> gbatch_launch_desc(bte_batch *bt, BatchState<real> &bs, const bte_batch::Cls &c, int tid, int parity) {
    SweepBatch<real> d{};
    d.params = bs.gsweep[parity].template as<SweepParams<real>>();
    d.inst = bt->d_inst.as<int>() + c.begin;
    d.n_inst = c.count;
    d.chunks = (int)ws_of<real>(bt->plans[bt->inst[c.begin]]).subsets.at(tid).first.size();
    for (int q = 1; q < c.count; ++q)
        d.chunks = std::max(d.chunks, (int)ws_of<real>(bt->plans[bt->inst[c.begin + q]]).subsets.at(tid).first.size());
    d.B = bt->plans[bt->inst[c.begin]]->B;
    d.WY = c.nrb;
    d.R_max = c.R_max;
    return d;
}

// one class's sweep launch
template <typename real>
cudaError_t batch_class_sweep(bte_batch *bt, BatchState<real> &bs, const bte_batch::Cls &c, int tid, int parity,
                              cudaStream_t s) {
    if (c.general) return launch_sweep_batch<real>(gbatch_launch_desc(bt, bs, c, tid, parity), tile_of(tid).dw, s);
    return launch_sweep2dp_batch<real>(batch_launch_desc(bt, bs, c, tid, parity), tile_of(tid).dw, s);
}

// Per-instance launch parameters of every class's tile, both parities.
template <typename real>
int batch_upload_params(bte_batch *bt, BatchState<real> &bs, const std::vector<int> &tiles, double tol) {
    std::vector<Sweep2DParams<real>> sw((size_t)bt->n);
    std::vector<SweepParams<real>> gsw((size_t)bt->n);
    std::vector<UpdateParams<real>> up((size_t)bt->n);
    Status *st_all = bt->d_status.as<Status>();
    for (int par = 0; par < 2; ++par) {
        for (size_t c = 0; c < bt->classes.size(); ++c) {
            const bte_batch::Cls &cl = bt->classes[c];
            for (int q = 0; q < cl.count; ++q) {
                const int i = bt->inst[cl.begin + q];
                bte_plan *p = bt->plans[i];
                Workspace<real> &ws = ws_of<real>(p);
                const int tid = tiles[c];
                if (int rc = ensure_subsets(p, ws, tid)) return bfail(bt, rc, p->err);
                if (cl.general) {
                    SweepParams<real> gp = sweep_params(p, ws, tid, false);
                    gp.tsrc = ws.tdev[par].template as<real>();
                    gp.ein = ws.ein[par].template as<real>();
                    gp.ein_smem = 0;
                    gp.store_e = 0;
                    gp.e = nullptr;
                    gp.done = &st_all[i].done;
                    gsw[i] = gp;
                }
                Sweep2DParams<real> sp = sweep2d_params(p, ws, tid, false);
                sp.tsrc = ws.tdev[par].template as<real>();
                sp.ein = ws.ein[par].template as<real>();
                sp.store_e = 0;
                sp.e = nullptr;
                sp.done = &st_all[i].done;
                sp.status = &st_all[i].status;
                FinalizeParams fin = fin_params(p, tol, false);
                fin.nblocks = update_cell_block_count(p->N, upd_vec_batch(p));
                fin.done = &st_all[i].done;
                fin.iter = &st_all[i].iter;
                fin.status = &st_all[i].status;
                fin.pending = &st_all[i].pending;
                fin.last = st_all[i].last;
                fin.batch_done = bt->d_done.as<int>();
                sp.fin = fin;
                sw[i] = sp;
                UpdateParams<real> u = update_params(p, ws, tid, false, tol);
                u.vec = upd_vec_batch(p) ? 1 : 0;
                u.x_in = ws.T[par].template as<double>();
                u.x_out = ws.T[par ^ 1].template as<double>();
                u.xdev_out = ws.tdev[par ^ 1].template as<real>();
                u.ein_out = ws.ein[par ^ 1].template as<real>();
                u.done = &st_all[i].done;
                u.iter = &st_all[i].iter;
                u.status = &st_all[i].status;
                u.last = st_all[i].last;
                u.batch_done = bt->d_done.as<int>();
                u.fin = sp.fin;
                // row-pipeline sweeps finalize in their prologue; the general
                // kernel's instances finalize in the update itself
                u.defer = cl.general ? 0 : 1;
                up[i] = u;
            }
        }
        BCK(bt, bs.sweep[par].ensure(sizeof(Sweep2DParams<real>) * bt->n));
        BCK(bt, bs.gsweep[par].ensure(sizeof(SweepParams<real>) * bt->n));
        BCK(bt, bs.update[par].ensure(sizeof(UpdateParams<real>) * bt->n));
        BCK(bt, cudaMemcpy(bs.sweep[par].p, sw.data(), sizeof(Sweep2DParams<real>) * bt->n, cudaMemcpyHostToDevice));
        BCK(bt, cudaMemcpy(bs.gsweep[par].p, gsw.data(), sizeof(SweepParams<real>) * bt->n, cudaMemcpyHostToDevice));
        BCK(bt, cudaMemcpy(bs.update[par].p, up.data(), sizeof(UpdateParams<real>) * bt->n, cudaMemcpyHostToDevice));
    }
    return BTE_OK;
}

// One batched iteration: the class sweeps (concurrently on the side streams,
// joined back into `stream`), then one update launch over every instance.
template <typename real>
cudaError_t batch_enqueue(bte_batch *bt, BatchState<real> &bs, const std::vector<int> &tiles, int parity,
                          cudaStream_t stream, bool timed = false) {
    cudaError_t e = timed ? record_timing_event(bt->tev[0], stream) : cudaSuccess;
    if (e == cudaSuccess) e = cudaEventRecord(bt->fork, stream);
    for (size_t c = 0; c < bt->classes.size() && e == cudaSuccess; ++c) {
        cudaStream_t s = bt->side[c];
        e = cudaStreamWaitEvent(s, bt->fork, 0);
        if (e == cudaSuccess) e = batch_class_sweep<real>(bt, bs, bt->classes[c], tiles[c], parity, s);
        if (e == cudaSuccess) e = cudaEventRecord(bt->join[c], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, bt->join[c], 0);
    }
    if (e == cudaSuccess && timed) e = record_timing_event(bt->tev[1], stream);
    if (e != cudaSuccess) return e;
    return launch_update_batch<real>(bs.update[parity].template as<UpdateParams<real>>(), bt->d_table.as<int2>(),
                                     bt->upd_blocks, stream);
}

template <typename real>
int batch_solve_t(bte_batch *bt, const bte_solve_opts *o, double *T_out, bte_stats *st, bte_batch_stats *bst) {
    cudaStream_t stream = (cudaStream_t)o->stream;
    BatchState<real> &bs = bstate_of<real>(bt);
    if (o->T_wall) return bfail(bt, BTE_EINVAL, "bte_batch_solve: wall temperatures come from each instance's plan");
    if (o->tile_kind != 0 && o->tile_kind != 3)
        return bfail(bt, BTE_EINVAL, "bte_batch_solve: the batch picks its kernels (tile_kind 0 or 3)");
    // per-instance state
    for (int i = 0; i < bt->n; ++i) {
        bte_plan *p = bt->plans[i];
        Workspace<real> &ws = ws_of<real>(p);
        if (int rc = ensure_workspace(p, ws)) return bfail(bt, rc, p->err);
        p->cur_tau = p->tau;
        if (o->tau) {
            for (int b = 0; b < p->B; ++b)
                if (!(o->tau[b] > 0.0) || !std::isfinite(o->tau[b])) return bfail(bt, BTE_EINVAL, "tau override must be > 0");
            p->cur_tau.assign(o->tau, o->tau + p->B);
        }
        p->cur_Tw.assign(p->bc_T, p->bc_T + 6);
        p->cur_Q = o->Q_amp_each ? o->Q_amp_each[i] : o->Q_amp;
        if (int rc = begin_state(p, o, ws, stream)) return bfail(bt, rc, p->err);
        if (int rc = upload_tables(p, ws)) return bfail(bt, rc, p->err);
        p->solved = false;  // a batch solve leaves no adjoint-ready state in the plans
    }
    BCK(bt, cudaMemsetAsync(bt->d_status.p, 0, sizeof(Status) * bt->n, stream));
    BCK(bt, cudaMemsetAsync(bt->d_done.p, 0, sizeof(int), stream));
    const double tol = o->tol;
    // tiles: per class, the caller's restriction, then the autotuned choice (cached)
    const std::vector<int> req = {o->dirs_per_lane, o->dirs_per_cta};
    std::vector<int> tiles;
    if (bs.tuned.count(req)) {
        tiles = bs.tuned[req];
    } else {
        for (size_t c = 0; c < bt->classes.size(); ++c) {
            std::vector<int> cand = batch_class_candidates(bt, bt->classes[c], (int)sizeof(real), o->dirs_per_lane,
                                                           o->dirs_per_cta);
            if (cand.empty()) return bfail(bt, BTE_EINVAL, "no sweep tile fits a size class of the batch");
            tiles.push_back(cand[0]);
        }
        for (size_t c = 0; c < bt->classes.size(); ++c) {
            std::vector<int> cand = batch_class_candidates(bt, bt->classes[c], (int)sizeof(real), o->dirs_per_lane,
                                                           o->dirs_per_cta);
            if (cand.size() == 1) continue;
            float best = 1e30f;
            for (int tid : cand) {
                std::vector<int> trial = tiles;
                trial[c] = tid;
                if (int rc = batch_upload_params<real>(bt, bs, trial, 0.0)) return rc;
                float tmin = 1e30f;
                for (int rep = 0; rep < 4; ++rep) {
                    cudaEventRecord(bt->ev0, stream);
                    cudaError_t e = batch_class_sweep<real>(bt, bs, bt->classes[c], tid, 0, stream);
                    cudaEventRecord(bt->ev1, stream);
                    cudaEventSynchronize(bt->ev1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, bt->ev0, bt->ev1);
                    if (e != cudaSuccess) {
                        cudaGetLastError();
                        tmin = 1e30f;
                        break;
                    }
                    if (rep >= 1) tmin = std::min(tmin, ms);
                }
                if (std::getenv("BTE_TUNE_VERBOSE"))
                    std::fprintf(stderr, "bte batch tune: class nrb %d dw %d cw %d: %.4f ms\n", bt->classes[c].nrb,
                                 tile_of(tid).dw, tile_of(tid).cw, tmin);
                if (tmin < best) {
                    best = tmin;
                    tiles[c] = tid;
                }
            }
        }
        bs.tuned[req] = tiles;
        // autotuning ran sweeps on the initial state: start again
        for (int i = 0; i < bt->n; ++i) {
            bte_plan *p = bt->plans[i];
            if (int rc = begin_state(p, o, ws_of<real>(p), stream)) return bfail(bt, rc, p->err);
        }
        BCK(bt, cudaMemsetAsync(bt->d_status.p, 0, sizeof(Status) * bt->n, stream));
        BCK(bt, cudaMemsetAsync(bt->d_done.p, 0, sizeof(int), stream));
    }
    if (int rc = batch_upload_params<real>(bt, bs, tiles, tol)) return rc;
    int poll = o->poll_every > 0 ? o->poll_every : 32;
    poll = std::max(2, poll + (poll & 1));
    std::vector<int> key = tiles;
    key.push_back(poll);
    key.push_back(bt->time_sweeps ? 1 : 0);
    key.push_back((int)(tol * 1e15 > 2e9 ? 2e9 : tol * 1e15));
    if (!bs.graph || bs.graph_key != key) {
        if (bs.graph) {
            cudaGraphExecDestroy(bs.graph);
            bs.graph = nullptr;
        }
        // one batched iteration outside any capture sets the kernels'
        // shared-memory attributes; then the state starts again
        BCK(bt, batch_enqueue<real>(bt, bs, tiles, 0, stream));
        for (int i = 0; i < bt->n; ++i) {
            bte_plan *p = bt->plans[i];
            if (int rc = begin_state(p, o, ws_of<real>(p), stream)) return bfail(bt, rc, p->err);
        }
        BCK(bt, cudaMemsetAsync(bt->d_status.p, 0, sizeof(Status) * bt->n, stream));
        BCK(bt, cudaMemsetAsync(bt->d_done.p, 0, sizeof(int), stream));
        cudaStream_t cs;
        BCK(bt, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g;
        cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        for (int i = 0; i < poll && ce == cudaSuccess; ++i)
            ce = batch_enqueue<real>(bt, bs, tiles, i & 1, cs, bt->time_sweeps && i == 0);
        if (ce == cudaSuccess) ce = launch_finalize<real>(bs.update[0].template as<UpdateParams<real>>(), bt->n, cs);
        cudaError_t ce2 = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (ce != cudaSuccess) return bfail(bt, BTE_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(ce));
        if (ce2 != cudaSuccess) return bfail(bt, BTE_ECUDA, std::string("batch graph capture end: ") + cudaGetErrorString(ce2));
        ce = cudaGraphInstantiate(&bs.graph, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) {
            bs.graph = nullptr;
            return bfail(bt, BTE_ECUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(ce));
        }
        bs.graph_key = key;
    }
    const int max_iter = o->max_iter;
    int enq = 0;
    long long launches = 0;
    double sweep_ms = 0.0;
    long long n_timed = 0;
    BCK(bt, cudaEventRecord(bt->ev0, stream));
    while (enq < max_iter) {
        const int k = std::min(poll, max_iter - enq);
        if (k == poll) {
            BCK(bt, cudaGraphLaunch(bs.graph, stream));
        } else {
            for (int i = 0; i < k; ++i)
                BCK(bt, batch_enqueue<real>(bt, bs, tiles, (enq + i) & 1, stream, bt->time_sweeps && i == 0));
            BCK(bt, launch_finalize<real>(bs.update[0].template as<UpdateParams<real>>(), bt->n, stream));
        }
        enq += k;
        launches += (long long)k * (long long)(bt->classes.size() + 1) + 1;
        BCK(bt, cudaMemcpyAsync(bt->h_done, bt->d_done.p, sizeof(int), cudaMemcpyDeviceToHost, stream));
        BCK(bt, cudaStreamSynchronize(stream));
        if (bt->time_sweeps) {
            float t = 0.f;
            BCK(bt, cudaEventElapsedTime(&t, bt->tev[0], bt->tev[1]));
            sweep_ms += t;
            n_timed += 1;
        }
        if (*bt->h_done >= bt->n) break;
    }
    BCK(bt, cudaEventRecord(bt->ev1, stream));
    BCK(bt, cudaEventSynchronize(bt->ev1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, bt->ev0, bt->ev1);
    std::vector<Status> hs((size_t)bt->n);
    BCK(bt, cudaMemcpy(hs.data(), bt->d_status.p, sizeof(Status) * bt->n, cudaMemcpyDeviceToHost));
    long long off = 0;
    double updates = 0.0;
    int n_conv = 0, max_it = 0, n_bad = 0;
    for (int i = 0; i < bt->n; ++i) {
        bte_plan *p = bt->plans[i];
        Workspace<real> &ws = ws_of<real>(p);
        const int it = hs[i].iter;
        BCK(bt, cudaMemcpyAsync(T_out + off, ws.T[it & 1].p, sizeof(double) * p->N, cudaMemcpyDefault, stream));
        off += p->N;
        updates += (double)it * p->n_active * p->B * p->D;
        const bool bad = hs[i].status != 0;
        const bool conv = tol > 0.0 && hs[i].done && !bad;
        n_conv += conv ? 1 : 0;
        n_bad += bad ? 1 : 0;
        max_it = std::max(max_it, it);
        if (st) {
            bte_stats &s = st[i];
            std::memset(&s, 0, sizeof(s));
            s.eps_q = NAN;
            s.iterations = it;
            s.converged = conv ? 1 : 0;
            s.eps_T = hs[i].last[0];
            s.T_max = hs[i].last[1];
            s.seconds = ms * 1e-3;
            const int ci = [&] {
                for (size_t c = 0; c < bt->classes.size(); ++c) {
                    const bte_batch::Cls &cl = bt->classes[c];
                    for (int q = 0; q < cl.count; ++q)
                        if (bt->inst[cl.begin + q] == i) return (int)c;
                }
                return 0;
            }();
            s.dirs_per_lane = tile_of(tiles[ci]).dw;
            s.dirs_per_cta = tile_of(tiles[ci]).cw;
            s.tile_kind = abi_kind(tile_of(tiles[ci]).kind);
            s.source_staged = tile_of(tiles[ci]).kind == 4 ? 0 : 1;
        }
    }
    BCK(bt, cudaStreamSynchronize(stream));
    if (bst) {
        std::memset(bst, 0, sizeof(*bst));
        bst->instances = bt->n;
        bst->converged = n_conv;
        bst->max_iterations = max_it;
        bst->seconds = ms * 1e-3;
        bst->updates = updates;
        bst->updates_per_s = ms > 0 ? updates / (ms * 1e-3) : 0.0;
        bst->kernel_launches = launches;
        bst->classes = (int)bt->classes.size();
        bst->sweep_seconds = sweep_ms * 1e-3;
        bst->sweep_iterations = n_timed;
    }
    for (int i = 0; i < bt->n; ++i)
        if (hs[i].status == 2) return bfail(bt, BTE_ETIMEOUT, "a bounded device wait expired in a batched sweep");
    if (n_bad) return bfail(bt, BTE_ENUMERIC, "NaN or Inf in the temperature update of an instance");
    if (tol > 0.0 && n_conv < bt->n) return bfail(bt, BTE_ENOTCONVERGED, "max_iter reached before every instance converged");
    return BTE_OK;
}
}  // namespace

namespace bte {
// Error text for calls without a plan (read back by bte_last_error(NULL)).
void set_global_error(const std::string &msg) { g_create_error = msg; }
}  // namespace bte

// ---------------------------------------------------------------------------
// Sharded solves of one instance (bands split over ranks).  Every outer
// iteration of the paper's solution procedure needs, per cell, the sum over
// all bands of the band-weighted direction sums (the temperature update);
// each band's sweep and its diffuse inflow depend only on T and on that
// band.  So a rank sweeps its bands and forms their weighted sum W_r (and its
// bands' next inflow), the ranks add their W_r (one FP64 allreduce of N
// values per iteration), and every rank forms the same T from the sum.
// ---------------------------------------------------------------------------
template <typename real>
int shard_begin_t(bte_plan *p, const bte_solve_opts *o) {
    cudaStream_t stream = (cudaStream_t)o->stream;
    Workspace<real> &ws = ws_of<real>(p);
    int rc = ensure_workspace(p, ws);
    if (rc) return rc;
    p->cur_tau = p->tau;
    if (o->tau) {
        for (int b = 0; b < p->B; ++b)
            if (!(o->tau[b] > 0.0) || !std::isfinite(o->tau[b])) return fail(p, BTE_EINVAL, "tau override must be > 0");
        p->cur_tau.assign(o->tau, o->tau + p->B);
    }
    p->cur_Tw.assign(p->bc_T, p->bc_T + 6);
    if (o->T_wall) p->cur_Tw.assign(o->T_wall, o->T_wall + 6);
    p->cur_Q = o->Q_amp;
    if ((rc = begin_state(p, o, ws, stream))) return rc;
    if ((rc = upload_tables(p, ws))) return rc;
    std::vector<int> cand = tile_candidates(p, (int)sizeof(real), o->tile_kind, o->dirs_per_lane, o->dirs_per_cta,
                                            o->source_staging, o->warps_z, o->lane_axis);
    if (cand.empty()) return fail(p, BTE_EINVAL, "no sweep tile supports this grid / tile request");
    // the tile a solve of this plan autotuned in this precision, else the first candidate
    int tid = cand[0];
    if (p->solved_precision == (sizeof(real) == 4 ? BTE_FP32 : BTE_FP64) &&
        std::find(cand.begin(), cand.end(), p->solved_tile) != cand.end())
        tid = p->solved_tile;
    if ((rc = ensure_subsets(p, ws, tid))) return rc;
    CK(p, ws.wsum.ensure(sizeof(double) * p->N));
    CK(p, cudaMemsetAsync(p->d_status.p, 0, sizeof(Status), stream));
    CK(p, cudaMemsetAsync(p->d_counter.p, 0, sizeof(unsigned int), stream));
    CK(p, cudaStreamSynchronize(stream));
    p->stream = stream;
    p->shard_prec = sizeof(real) == 4 ? BTE_FP32 : BTE_FP64;
    p->shard_tile = tid;
    p->shard_par = 0;
    p->shard_iters = 0;
    return BTE_OK;
}

template <typename real>
int shard_sweep_t(bte_plan *p, int b0, int b1, double *W_out) {
    Workspace<real> &ws = ws_of<real>(p);
    cudaStream_t stream = p->stream;
    const int par = p->shard_par, tid = p->shard_tile;
    CK(p, launch_tile_sweep<real>(p, ws, tid, false, ws.tdev[par].template as<real>(), ws.ein[par].template as<real>(),
                                  false, false, stream, nullptr, nullptr, nullptr, b0, b1 - b0));
    UpdateParams<real> u = update_params(p, ws, tid, false, 0.0);
    u.vec = 0;
    u.defer = 0;
    u.ignore_done = 1;
    u.ub0 = b0;
    u.ub1 = b1;
    u.w_out = ws.wsum.template as<double>();
    u.x_in = ws.T[par].template as<double>();
    u.ein_out = ws.ein[par ^ 1].template as<real>();   // this rank's bands' next inflow
    CK(p, launch_update<real>(u, stream));
    CK(p, cudaMemcpyAsync(W_out, ws.wsum.p, sizeof(double) * p->N, cudaMemcpyDefault, stream));
    CK(p, cudaStreamSynchronize(stream));
    return BTE_OK;
}

template <typename real>
int shard_apply_t(bte_plan *p, const double *W, double *T_out, double *eps_T) {
    Workspace<real> &ws = ws_of<real>(p);
    cudaStream_t stream = p->stream;
    const int par = p->shard_par, tid = p->shard_tile;
    CK(p, cudaMemcpyAsync(ws.wsum.p, W, sizeof(double) * p->N, cudaMemcpyDefault, stream));
    UpdateParams<real> u = update_params(p, ws, tid, false, 0.0);
    u.vec = 0;
    u.defer = 0;
    u.ignore_done = 1;
    u.fin.nblocks = update_cell_block_count(p->N, false);
    u.eps_hist = nullptr;
    u.x_in = ws.T[par].template as<double>();
    u.x_out = ws.T[par ^ 1].template as<double>();
    u.xdev_out = ws.tdev[par ^ 1].template as<real>();
    if (is_pipe3(tile_of(tid).kind)) u.xskew_out = ws.skt[pipe3_map(tile_of(tid))][par ^ 1].template as<real>();
    CK(p, launch_apply<real>(u, ws.wsum.template as<double>(), stream));
    CK(p, cudaMemcpyAsync(p->h_status, p->d_status.p, sizeof(Status), cudaMemcpyDeviceToHost, stream));
    if (T_out) CK(p, cudaMemcpyAsync(T_out, ws.T[par ^ 1].p, sizeof(double) * p->N, cudaMemcpyDefault, stream));
    CK(p, cudaStreamSynchronize(stream));
    p->shard_par ^= 1;
    ++p->shard_iters;
    if (eps_T) *eps_T = p->h_status->last[0];
    if (!std::isfinite(p->h_status->last[0])) return fail(p, BTE_ENUMERIC, "NaN or Inf in the sharded temperature");
    return BTE_OK;
}

namespace {
template <typename real>
int get_state_t(bte_plan *p, double *T_out, double *ein_out) {
    Workspace<real> &ws = ws_of<real>(p);
    const int par = p->solved_iters & 1;   // the state set the next iteration would read
    CK(p, cudaStreamSynchronize(p->stream));
    if (T_out) CK(p, cudaMemcpy(T_out, ws.T[par].p, sizeof(double) * p->N, cudaMemcpyDefault));
    if (ein_out && p->F > 0) {
        const int B = p->B, F = p->F;
        std::vector<real> e((size_t)B * F);
        CK(p, cudaMemcpy(e.data(), ws.ein[par].p, sizeof(real) * e.size(), cudaMemcpyDeviceToHost));
        std::vector<double> out(e.size());
        for (int b = 0; b < B; ++b)
            for (int f = 0; f < F; ++f)
                out[(size_t)b * F + f] = (double)e[(size_t)b * F + f] + p->C[b] * p->T_ref / kFourPi;
        CK(p, cudaMemcpy(ein_out, out.data(), sizeof(double) * out.size(), cudaMemcpyDefault));
    }
    return BTE_OK;
}
}  // namespace

extern "C" {

const char *bte_version(void) { return "libbte 0.1 (sm_103a)"; }

void bte_default_opts(bte_solve_opts *o) {
    std::memset(o, 0, sizeof(*o));
    o->precision = BTE_FP32;
    o->tol = 1e-6;
    o->max_iter = 100000;
    o->T_init = nullptr;
    o->T_init_uniform = 300.0;
    o->Q_amp = 1.0;
    o->poll_every = 32;
}

namespace {
// Debug mode: every index table of a plan checked against its extent before
// upload (the message of the first violation, or null).
const char *validate_tables(const bte_plan *p) {
    const long long N = p->N;
    const int F = p->F, D = p->D;
    if ((long long)p->face_cell.size() != F || (int)p->face_side.size() != F || (int)p->face_kind.size() != F)
        return "face table sizes differ from the face count";
    for (int f = 0; f < F; ++f) {
        if (p->face_cell[f] < 0 || p->face_cell[f] >= N || !p->mask[p->face_cell[f]]) return "face cell outside the solid";
        if (p->face_side[f] < 0 || p->face_side[f] >= 2 * p->dim) return "face side outside 0 .. 2 dim";
        if (p->face_kind[f] < 0 || p->face_kind[f] > 2) return "face kind outside 0 .. 2";
    }
    for (long long c = 0; c < N; ++c) {
        const int base = p->cellinfo[c].x, flags = p->cellinfo[c].y;
        const unsigned bm = ((unsigned)flags >> kSideShift) & 63u;
        if (base < 0 || base + __builtin_popcount(bm) > F) return "cell face base outside the face table";
        for (int side = 0; side < 6; ++side) {
            if (!((bm >> side) & 1u)) continue;
            const int f = face_of(base, flags, side);
            if (p->face_cell[f] != c || p->face_side[f] != side) return "cell face index does not point at its face";
            if ((((unsigned)flags >> (kSpecShift + side)) & 1u) != (p->face_kind[f] == 2 ? 1u : 0u))
                return "specular flag of a cell side differs from its face kind";
        }
    }
    for (int v : p->wall_face)
        if (v < -1 || v >= F) return "wall face index outside the face table";
    std::vector<int> seen(D, 0);
    for (int d : p->perm) {
        if (d < 0 || d >= D || seen[d]++) return "direction permutation is not a permutation";
    }
    for (int v : p->sidx)
        if (v < -1 || v >= p->Fs) return "specular face index outside 0 .. Fs";
    for (int v : p->mirror)
        if (v < -1 || v >= D) return "mirror direction outside 0 .. D";
    return nullptr;
}
}  // namespace

int bte_create(const bte_grid *g, const uint8_t *mask, const bte_bands *bands, const bte_quad *quad,
               const bte_bcs *bcs, const double *q_profile, bte_plan **out) {
    NvtxRange nvtx_range("bte_create");
    if (!out) return fail(nullptr, BTE_EINVAL, "out is null");
    *out = nullptr;
    std::unique_ptr<bte_plan> p(new (std::nothrow) bte_plan());
    if (!p) return fail(nullptr, BTE_ENOMEM, "host allocation failed");
    int rc = build_plan(p.get(), g, mask, bands, quad, bcs, q_profile);
    if (rc) return rc;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) return fail(nullptr, BTE_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(ce));
#define CKC(expr)                                                                                               \
    do {                                                                                                        \
        cudaError_t _e = (expr);                                                                                \
        if (_e != cudaSuccess)                                                                                  \
            return fail(nullptr, _e == cudaErrorMemoryAllocation ? BTE_ENOMEM : BTE_ECUDA,                      \
                        std::string(#expr) + ": " + cudaGetErrorString(_e));                                    \
    } while (0)
    if (debug_mode())
        if (const char *m = validate_tables(p.get())) return fail(nullptr, BTE_ECORRUPT, std::string("debug mode: ") + m);
    CKC(upload(p->d_cell, p->cellinfo));
    CKC(upload(p->d_face_cell, p->face_cell));
    CKC(upload(p->d_face_side, p->face_side));
    CKC(upload(p->d_face_kind, p->face_kind));
    CKC(upload(p->d_perm, p->perm));
    if (p->Fs > 0) {
        CKC(upload(p->d_sidx, p->sidx));
        CKC(upload(p->d_mirror, p->mirror));
    }
    CKC(upload(p->d_dneg, p->dneg));
    CKC(upload(p->ws32.wall, p->wall_face));
    CKC(upload(p->ws64.wall, p->wall_face));
    CKC(p->d_status.ensure(sizeof(Status)));
    CKC(p->d_counter.ensure(sizeof(unsigned int)));
    CKC(cudaMemset(p->d_counter.p, 0, sizeof(unsigned int)));
    const long long nblk = (p->N + 31) / 32 + ((long long)std::max(p->F, 1) * p->B + 255) / 256 + 16;
    CKC(p->d_blockpart.ensure(sizeof(double) * 2 * nblk));
    p->hist_cap = 1 << 16;
    CKC(p->d_hist.ensure(sizeof(double) * p->hist_cap));
    CKC(cudaMallocHost(&p->h_status, sizeof(Status)));
    CKC(cudaEventCreate(&p->ev0));
    CKC(cudaEventCreate(&p->ev1));
#undef CKC
    *out = p.release();
    return BTE_OK;
}

int bte_solve(bte_plan *p, const bte_solve_opts *o, double *T_out, double *q_out, void *e_out, bte_stats *st) {
    NvtxRange nvtx_range("bte_solve");
    if (!p) return fail(nullptr, BTE_EINVAL, "plan is null");
    if (!o || !T_out) return fail(p, BTE_EINVAL, "opts and T_out are required");
    if (o->max_iter < 1) return fail(p, BTE_EINVAL, "max_iter must be >= 1");
    if (!o->T_init && !(o->T_init_uniform > 0.0)) return fail(p, BTE_EINVAL, "T_init_uniform must be > 0");
    if (!std::isfinite(o->Q_amp)) return fail(p, BTE_EINVAL, "Q_amp must be finite");
    if (o->Q_amp_each) return fail(p, BTE_EINVAL, "Q_amp_each is for batched solves");
    if (o->ein_init && !o->T_init) return fail(p, BTE_EINVAL, "ein_init resumes a state: it needs T_init");
    if (o->T_wall)
        for (int f = 0; f < 6; ++f)
            if (f / 2 < p->dim && p->bc_type[f] == BTE_BC_ISOTHERMAL && (!(o->T_wall[f] > 0) || !std::isfinite(o->T_wall[f])))
                return fail(p, BTE_EINVAL, "T_wall override must be > 0");
    if (o->face_order < 0 || o->face_order > 2) return fail(p, BTE_EINVAL, "face_order must be 0, 1 or 2");
    p->solved = false;
    p->xmode = o->face_order == 2 ? 2 : 0;
    p->cur_inv_dt = 0.0;
    p->forced_T_ref = NAN;
    int rc;
    if (o->precision == BTE_FP32)
        rc = solve_t<float>(p, o, T_out, q_out, e_out, st);
    else if (o->precision == BTE_FP64)
        rc = solve_t<double>(p, o, T_out, q_out, e_out, st);
    else
        rc = fail(p, BTE_EINVAL, "precision must be BTE_FP32 or BTE_FP64");
    p->xmode = 0;
    return guard_rc(p, rc);
}

int bte_adjoint_ex(bte_plan *p, const double *dJ_dT, double tol, int max_iter, double *g_tau, double *g_Twall,
                   double *g_Qamp, double *g_L, bte_stats *st) {
    NvtxRange nvtx_range("bte_adjoint_ex");
    if (!p) return fail(nullptr, BTE_EINVAL, "plan is null");
    if (!dJ_dT) return fail(p, BTE_EINVAL, "dJ_dT is required");
    if (max_iter < 1) return fail(p, BTE_EINVAL, "max_iter must be >= 1");
    if (!p->solved || p->solved_iters < 1) return fail(p, BTE_ESTATE, "bte_adjoint needs a preceding bte_solve");
    if (p->solved_order != 1)
        return fail(p, BTE_ESTATE, "bte_adjoint differentiates step-face solves (face_order 1) only");
    p->want_glen = g_L != nullptr;
    const int rc = p->solved_precision == BTE_FP32
                       ? adjoint_t<float>(p, dJ_dT, tol, max_iter, g_tau, g_Twall, g_Qamp, g_L, st)
                       : adjoint_t<double>(p, dJ_dT, tol, max_iter, g_tau, g_Twall, g_Qamp, g_L, st);
    p->want_glen = false;
    return guard_rc(p, rc);
}

int bte_adjoint(bte_plan *p, const double *dJ_dT, double tol, int max_iter, double *g_tau, double *g_Twall,
                double *g_Qamp, bte_stats *st) {
    return bte_adjoint_ex(p, dJ_dT, tol, max_iter, g_tau, g_Twall, g_Qamp, nullptr, st);
}

int bte_transient(bte_plan *p, const bte_solve_opts *o, double dt, int n_steps, double *T_out, double *T_hist,
                  bte_stats *st) {
    NvtxRange nvtx_range("bte_transient");
    if (!p) return fail(nullptr, BTE_EINVAL, "plan is null");
    if (!o || !T_out) return fail(p, BTE_EINVAL, "opts and T_out are required");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(p, BTE_EINVAL, "dt must be finite and > 0");
    if (n_steps < 1) return fail(p, BTE_EINVAL, "n_steps must be >= 1");
    if (o->max_iter < 1) return fail(p, BTE_EINVAL, "max_iter must be >= 1");
    if (o->face_order == 2) return fail(p, BTE_EINVAL, "transient steps use step faces (face_order 0 or 1)");
    if (o->face_order < 0 || o->face_order > 2) return fail(p, BTE_EINVAL, "face_order must be 0, 1 or 2");
    if (o->tile_kind != 0 && o->tile_kind != 1 && !(o->tile_kind == 3 && p->dim == 3))
        return fail(p, BTE_EINVAL, "transient steps use the general kernel (or, on 3D grids, the plane pipeline)");
    if (!o->T_init && !(o->T_init_uniform > 0.0)) return fail(p, BTE_EINVAL, "T_init_uniform must be > 0");
    if (!std::isfinite(o->Q_amp)) return fail(p, BTE_EINVAL, "Q_amp must be finite");
    if (o->Q_amp_each) return fail(p, BTE_EINVAL, "Q_amp_each is for batched solves");
    if (o->T_wall)
        for (int f = 0; f < 6; ++f)
            if (f / 2 < p->dim && p->bc_type[f] == BTE_BC_ISOTHERMAL && (!(o->T_wall[f] > 0) || !std::isfinite(o->T_wall[f])))
                return fail(p, BTE_EINVAL, "T_wall override must be > 0");
    p->solved = false;
    int rc;
    if (o->precision == BTE_FP32)
        rc = transient_t<float>(p, o, dt, n_steps, T_out, T_hist, st);
    else if (o->precision == BTE_FP64)
        rc = transient_t<double>(p, o, dt, n_steps, T_out, T_hist, st);
    else
        rc = fail(p, BTE_EINVAL, "precision must be BTE_FP32 or BTE_FP64");
    p->xmode = 0;
    p->cur_inv_dt = 0.0;
    p->forced_T_ref = NAN;
    p->solved = false;   // no adjoint-ready state after a transient run
    return guard_rc(p, rc);
}


int bte_face_count(const bte_plan *p) { return p ? p->F : BTE_EINVAL; }

int bte_shard_begin(bte_plan *p, const bte_solve_opts *o) {
    if (!p) return fail(nullptr, BTE_EINVAL, "plan is null");
    if (!o) return fail(p, BTE_EINVAL, "opts are required");
    if (!o->T_init && !(o->T_init_uniform > 0.0)) return fail(p, BTE_EINVAL, "T_init_uniform must be > 0");
    if (!std::isfinite(o->Q_amp)) return fail(p, BTE_EINVAL, "Q_amp must be finite");
    if (o->Q_amp_each) return fail(p, BTE_EINVAL, "Q_amp_each is for batched solves");
    if (o->ein_init && !o->T_init) return fail(p, BTE_EINVAL, "ein_init resumes a state: it needs T_init");
    if (o->face_order == 2) return fail(p, BTE_EINVAL, "sharded solves use step faces (face_order 0 or 1)");
    if (p->Fs > 0) return fail(p, BTE_EINVAL, "sharded solves: specular faces carry per-direction state");
    if (o->tile_kind < 0 || o->tile_kind > 3) return fail(p, BTE_EINVAL, "tile_kind must be 0, 1, 2 or 3");
    p->solved = false;
    p->xmode = 0;
    p->cur_inv_dt = 0.0;
    p->forced_T_ref = NAN;
    p->shard_prec = -1;
    int rc;
    if (o->precision == BTE_FP32)
        rc = shard_begin_t<float>(p, o);
    else if (o->precision == BTE_FP64)
        rc = shard_begin_t<double>(p, o);
    else
        rc = fail(p, BTE_EINVAL, "precision must be BTE_FP32 or BTE_FP64");
    return guard_rc(p, rc);
}

int bte_shard_sweep(bte_plan *p, int b0, int b1, double *W_out) {
    NvtxRange nvtx_range("bte_shard_sweep");
    if (!p) return fail(nullptr, BTE_EINVAL, "plan is null");
    if (p->shard_prec < 0) return fail(p, BTE_ESTATE, "bte_shard_sweep needs bte_shard_begin");
    if (!W_out || b0 < 0 || b1 <= b0 || b1 > p->B) return fail(p, BTE_EINVAL, "need 0 <= b0 < b1 <= B and W_out");
    const int rc = p->shard_prec == BTE_FP32 ? shard_sweep_t<float>(p, b0, b1, W_out)
                                             : shard_sweep_t<double>(p, b0, b1, W_out);
    return guard_rc(p, rc);
}

int bte_shard_apply(bte_plan *p, const double *W, double *T_out, double *eps_T) {
    NvtxRange nvtx_range("bte_shard_apply");
    if (!p) return fail(nullptr, BTE_EINVAL, "plan is null");
    if (p->shard_prec < 0) return fail(p, BTE_ESTATE, "bte_shard_apply needs bte_shard_begin");
    if (!W) return fail(p, BTE_EINVAL, "W is required");
    const int rc = p->shard_prec == BTE_FP32 ? shard_apply_t<float>(p, W, T_out, eps_T)
                                             : shard_apply_t<double>(p, W, T_out, eps_T);
    return guard_rc(p, rc);
}

int bte_get_state(bte_plan *p, double *T_out, double *ein_out) {
    if (!p) return fail(nullptr, BTE_EINVAL, "plan is null");
    if (!p->solved || p->solved_iters < 1) return fail(p, BTE_ESTATE, "bte_get_state needs a preceding bte_solve");
    return p->solved_precision == BTE_FP32 ? get_state_t<float>(p, T_out, ein_out)
                                           : get_state_t<double>(p, T_out, ein_out);
}

int bte_profile_sweep(bte_plan *p, int reps, double *ms_per_sweep) {
    if (!p) return fail(nullptr, BTE_EINVAL, "plan is null");
    if (reps < 1 || !ms_per_sweep) return fail(p, BTE_EINVAL, "reps >= 1 and ms_per_sweep required");
    if (!p->solved || p->solved_iters < 1) return fail(p, BTE_ESTATE, "bte_profile_sweep needs a preceding bte_solve");
    if (p->solved_precision == BTE_FP32) return profile_t<float>(p, reps, ms_per_sweep);
    return profile_t<double>(p, reps, ms_per_sweep);
}

int bte_debug_overwrite_guard(bte_plan *p) {
    if (!p) return fail(nullptr, BTE_EINVAL, "plan is null");
    if (!debug_mode() || !p->d_status.guarded) return fail(p, BTE_ESTATE, "bte_debug_overwrite_guard: debug mode is off");
    // a host-side write into the allocation, just past the buffer's end
    const cudaError_t e = cudaMemset(static_cast<char *>(p->d_status.p) + p->d_status.bytes, 0, 1);
    if (e != cudaSuccess) return fail(p, BTE_ECUDA, cudaGetErrorString(e));
    return cudaDeviceSynchronize() == cudaSuccess ? BTE_OK : fail(p, BTE_ECUDA, "synchronisation failed");
}

int bte_debug_set_wait_limit(bte_plan *p, long long polls) {
    if (!p) return fail(nullptr, BTE_EINVAL, "plan is null");
    if (polls < 0) return fail(p, BTE_EINVAL, "bte_debug_set_wait_limit: polls must be >= 0");
    p->spin_limit = polls == 0 ? kPipeSpinLimit : polls;
    // captured graphs hold the old limit in their kernel parameters
    for (Workspace<float> *w : {&p->ws32}) {
        if (w->graph) cudaGraphExecDestroy(w->graph);
        if (w->agraph) cudaGraphExecDestroy(w->agraph);
        w->graph = w->agraph = nullptr;
    }
    for (Workspace<double> *w : {&p->ws64}) {
        if (w->graph) cudaGraphExecDestroy(w->graph);
        if (w->agraph) cudaGraphExecDestroy(w->agraph);
        w->graph = w->agraph = nullptr;
    }
    return BTE_OK;
}

int bte_set_sweep_timing(bte_plan *p, int every) {
    if (!p) return fail(nullptr, BTE_EINVAL, "plan is null");
    if (every < 0) return fail(p, BTE_EINVAL, "bte_set_sweep_timing: every must be >= 0");
    p->time_every = every;
    if (every && ensure_timing_events(p, 32) != cudaSuccess) {
        cudaGetLastError();
        p->time_every = 0;
        return fail(p, BTE_ECUDA, "bte_set_sweep_timing: cudaEventCreate failed");
    }
    return BTE_OK;
}

int bte_eps_history(const bte_plan *p, double *out, int n) {
    if (!p || !out || n < 0) return BTE_EINVAL;
    const int m = std::min(n, std::min(p->solved_iters, p->hist_cap));
    if (m > 0 && cudaMemcpy(out, p->d_hist.p, sizeof(double) * m, cudaMemcpyDeviceToHost) != cudaSuccess) return BTE_ECUDA;
    return m;
}

int bte_batch_create(int n, bte_plan *const *plans, bte_batch **out) {
    if (!out) return bfail(nullptr, BTE_EINVAL, "bte_batch_create: out is null");
    *out = nullptr;
    if (n < 1 || !plans) return bfail(nullptr, BTE_EINVAL, "bte_batch_create: n >= 1 plans required");
    for (int i = 0; i < n; ++i) {
        const bte_plan *p = plans[i];
        if (!p) return bfail(nullptr, BTE_EINVAL, "bte_batch_create: null plan");
        const bte_plan *q = plans[0];
        if (p->B != q->B || p->D != q->D)
            return bfail(nullptr, BTE_EINVAL, "bte_batch_create: every instance needs the same band and direction counts");
        if (p->dim > 2 || p->Fs > 0 || (p->ny + 31) / 32 > 32)
            return bfail(nullptr, BTE_EINVAL,
                         "bte_batch_create: instances must be 1D/2D grids of at most 1024 rows without specular faces");
        for (int j = 0; j < i; ++j)
            if (plans[j] == p) return bfail(nullptr, BTE_EINVAL, "bte_batch_create: a plan appears twice");
    }
    std::unique_ptr<bte_batch> bt(new bte_batch());
    bt->plans.assign(plans, plans + n);
    bt->n = n;
    // size classes by kernel and 32-row block count: unmasked single-region
    // instances of at most 16 row blocks run the row-pipeline kernel, the
    // others (masks, several regions) the general kernel; inside a class,
    // largest first
    auto rowpipe_ok_b = [](const bte_plan *p) { return p->n_active == p->N && p->R == 1 && (p->ny + 31) / 32 <= 16; };
    std::map<std::pair<int, int>, std::vector<int>> by;
    for (int i = 0; i < n; ++i) by[{rowpipe_ok_b(plans[i]) ? 0 : 1, (plans[i]->ny + 31) / 32}].push_back(i);
    for (auto &kv : by) {
        std::vector<int> v = kv.second;
        std::stable_sort(v.begin(), v.end(), [&](int a, int b) { return plans[a]->N > plans[b]->N; });
        bte_batch::Cls c{kv.first.second, (int)bt->inst.size(), (int)v.size(), 0, 0, kv.first.first, 1};
        for (int i : v) {
            c.nx_max = std::max(c.nx_max, plans[i]->nx);
            c.ny_max = std::max(c.ny_max, plans[i]->ny);
            c.R_max = std::max(c.R_max, plans[i]->R);
            bt->inst.push_back(i);
        }
        bt->classes.push_back(c);
    }
    // update blocks: largest classes first
    std::vector<int2> table;
    for (int ci = (int)bt->classes.size() - 1; ci >= 0; --ci) {
        const bte_batch::Cls &c = bt->classes[ci];
        for (int q = 0; q < c.count; ++q) {
            const int i = bt->inst[c.begin + q];
            const int nb = update_blocks(plans[i]->N, plans[i]->F, plans[i]->B, upd_vec_batch(plans[i]));
            for (int k = 0; k < nb; ++k) table.push_back(make_int2(i, k));
        }
    }
    bt->upd_blocks = (int)table.size();
    if (cudaSuccess != upload(bt->d_inst, bt->inst) || cudaSuccess != upload(bt->d_table, table) ||
        cudaSuccess != bt->d_status.ensure(sizeof(Status) * n) || cudaSuccess != bt->d_done.ensure(sizeof(int)) ||
        cudaSuccess != cudaMallocHost(&bt->h_done, sizeof(int)) || cudaSuccess != cudaEventCreate(&bt->fork) ||
        cudaSuccess != cudaEventCreate(&bt->ev0) || cudaSuccess != cudaEventCreate(&bt->ev1)) {
        cudaGetLastError();
        return bfail(nullptr, BTE_ECUDA, "bte_batch_create: device allocation failed");
    }
    for (size_t c = 0; c < bt->classes.size(); ++c) {
        cudaStream_t s;
        cudaEvent_t e;
        if (cudaSuccess != cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) return bfail(nullptr, BTE_ECUDA, "stream");
        bt->side.push_back(s);
        if (cudaSuccess != cudaEventCreateWithFlags(&e, cudaEventDisableTiming)) return bfail(nullptr, BTE_ECUDA, "event");
        bt->join.push_back(e);
    }
    *out = bt.release();
    return BTE_OK;
}

int bte_batch_solve(bte_batch *bt, const bte_solve_opts *o, double *T_out, bte_stats *st, bte_batch_stats *bs) {
    NvtxRange nvtx_range("bte_batch_solve");
    if (!bt) return bfail(nullptr, BTE_EINVAL, "batch is null");
    if (!o || !T_out) return bfail(bt, BTE_EINVAL, "opts and T_out are required");
    if (o->max_iter < 1) return bfail(bt, BTE_EINVAL, "max_iter must be >= 1");
    if (o->T_init || o->ein_init) return bfail(bt, BTE_EINVAL, "bte_batch_solve: use T_init_uniform (no T_init, ein_init)");
    if (o->face_order == 2) return bfail(bt, BTE_EINVAL, "bte_batch_solve: step faces only (face_order 0 or 1)");
    if (!std::isfinite(o->Q_amp)) return bfail(bt, BTE_EINVAL, "Q_amp must be finite");
    if (o->Q_amp_each)
        for (int i = 0; i < bt->n; ++i)
            if (!std::isfinite(o->Q_amp_each[i])) return bfail(bt, BTE_EINVAL, "Q_amp_each must be finite");
    int rc;
    if (o->precision == BTE_FP32)
        rc = batch_solve_t<float>(bt, o, T_out, st, bs);
    else if (o->precision == BTE_FP64)
        rc = batch_solve_t<double>(bt, o, T_out, st, bs);
    else
        return bfail(bt, BTE_EINVAL, "precision must be BTE_FP32 or BTE_FP64");
    if (debug_mode() && check_guards() != 0)
        return bfail(bt, BTE_ECORRUPT, "debug mode: a device buffer's guard words were overwritten");
    return rc;
}

int bte_batch_set_sweep_timing(bte_batch *bt, int on) {
    if (!bt) return bfail(nullptr, BTE_EINVAL, "batch is null");
    if (on) {
        for (cudaEvent_t &e : bt->tev)
            if (!e && cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                return bfail(bt, BTE_ECUDA, "bte_batch_set_sweep_timing: cudaEventCreate failed");
            }
    }
    bt->time_sweeps = on != 0;
    return BTE_OK;
}

void bte_batch_destroy(bte_batch *bt) { delete bt; }

const char *bte_batch_last_error(const bte_batch *bt) { return bt ? bt->err.c_str() : g_create_error.c_str(); }

void bte_destroy(bte_plan *p) { delete p; }

const char *bte_last_error(const bte_plan *p) { return p ? p->err.c_str() : g_create_error.c_str(); }

}  // extern "C"
