// Host side of the C ABI declared in include/geodock.h: context and device
// memory, topology checks and fragment tables (Alg. 1: the rotatable bonds
// and the two fragments on either side of each), run planning (work order,
// angle tables), the persistent batched launch in a CUDA graph, the plain
// one-launch-per-pair form, and the trace run.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <memory>
#include <numeric>
#include <string>
#include <tuple>
#include <thread>
#include <vector>

#include "../../include/geodock.h"
#define GD_DEFINE_AUX_KERNELS
#include "geodock_kernels.cuh"
#include "geodock_launch.h"
#include "geodock_refine_launch.h"

using namespace gd;

namespace {

// A named NVTX range over a scope (visible to a profiler's timeline; without one attached the calls do
// nothing).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    cudaError_t ensure(size_t bytes) {
        if (bytes <= n && p) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
        if (e == cudaSuccess) n = std::max<size_t>(bytes, 16);
        return e;
    }
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

// The padded field as a 3D texture (CUDA array, point sampling).
struct FieldTex {
    cudaArray_t arr = nullptr;
    cudaTextureObject_t tex = 0;
    ~FieldTex() {
        if (tex) cudaDestroyTextureObject(tex);
        if (arr) cudaFreeArray(arr);
    }
};

struct PocketH {
    bool live = false;
    PocketDev d{};
    std::unique_ptr<DevBuf> K;
    std::unique_ptr<FieldTex> Kt;
    std::unique_ptr<FieldTex> Kc;  // corner texture of the trilinear score
    std::unique_ptr<DevBuf> dev;  // device copy of d
    std::unique_ptr<DevBuf> pts;  // probe points for the exact score (float4, voxel + 0.5)
};

struct BatchH {
    bool live = false;
    int n = 0, natoms = 0, lmax = 1, nside_total = 0;
    int nidx = 0, ntor = 0, nchk = 0;  // sizes of the atom-index pool, torsion list and bump-pair rows
    std::vector<int> l, nside;            // per ligand
    std::vector<int> side_m, side_nmov, side_nfixB;  // per side
    std::vector<int> side_off;
    std::vector<int> atom_off;
    // every device array of the batch lives in one allocation
    std::unique_ptr<DevBuf> mem;
    LigDev* d_lig = nullptr;
    SideDev* d_side = nullptr;
    uint8_t* d_idx = nullptr;
    float* d_xyz0 = nullptr;
    // local refinement: torsions (side away from atom 0, deepest bond first) and bump-pair rows
    int tmax = 0;
    RefLigDev* d_rlig = nullptr;
    RefTorDev* d_rtor = nullptr;
    uint32_t* d_check = nullptr;
};

// Everything a batched run needs that depends on (batch, pockets, knobs, tile).
struct Plan {
    int ntask = 0, npairs = 0, slice = 0;
    std::vector<int> task_off;  // first task of each pair (plain form: pair order)
    std::unique_ptr<DevBuf> tasks, pockets, cs_hp, cs_lp, cs_peel, coarse;
    std::unique_ptr<DevBuf> skipped;  // per pair: pose-repetitions left out at a fixed point
    std::unique_ptr<DevBuf> looked;   // lookups left out by the gate (one u64)
    SweepParams P{};
    FinalParams F{};
    int kc = 12, Q = 1, W = 4, grid = 1, block = 128;
    size_t smem = 0;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t exec_stream = nullptr;
    ~Plan() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

}  // namespace

// Work of one repetition of one pose per ligand (from the topology and knobs)
// and the device counts of pose-repetitions the last run left out at a fixed
// point; dock_last_stats subtracts that work.
struct WorkTally {
    std::vector<uint64_t> cand, upd, bounds, pairs;
    int nlig = 0, npairs = 0;
    DevBuf* skipped = nullptr;
    DevBuf* looked = nullptr;
    bool pending = false;
};

// A ligand batch prepared on the host: the device arrays' contents and their
// places in one allocation.
struct BatchImage {
    std::vector<LigDev> lig;
    std::vector<RefLigDev> rlig;
    std::vector<SideDev> sides;
    std::vector<uint8_t> idx;
    std::vector<RefTorDev> rtor;
    std::vector<uint32_t> check;
    const float* xyz = nullptr;
    size_t o_lig = 0, o_side = 0, o_idx = 0, o_xyz = 0, o_rlig = 0, o_rtor = 0, o_chk = 0, total = 0;
};

// One stage of the database pipeline (dock_run_database): a chunk of ligands
// on the device with its plan, and pinned host memory for its upload and its
// results. Two of them alternate.
struct DbSlot {
    BatchH B;
    BatchImage im;
    std::unique_ptr<DevBuf> mem;
    Plan plan;
    std::vector<int32_t> aoff, boff, roff;  // the chunk's offsets, from 0
    void* stage = nullptr;
    void* hres = nullptr;
    void* hxyz = nullptr;
    void* hskip = nullptr;
    void* hlook = nullptr;
    size_t stage_bytes = 0, hres_bytes = 0, hxyz_bytes = 0, hskip_bytes = 0, hlook_bytes = 0;
    cudaEvent_t up = nullptr, done = nullptr;
    int c0 = 0, c1 = 0;
    bool pending = false;
    DbSlot() = default;
    DbSlot(const DbSlot&) = delete;
    DbSlot& operator=(const DbSlot&) = delete;
    ~DbSlot() {
        for (void* p : {stage, hres, hxyz, hskip, hlook})
            if (p) cudaFreeHost(p);
        if (up) cudaEventDestroy(up);
        if (done) cudaEventDestroy(done);
    }
};

struct dock_ctx {
    int device = 0;
    int num_sms = 1;
    std::string err;
    std::vector<PocketH> pockets;
    std::vector<BatchH> batches;
    dock_tile tile{0, 0, 0};           // forced shape (0 = automatic)
    std::map<std::string, dock_tile> tuned;  // autotuned shapes per (batch, knobs)
    DevBuf counter, pose_key, pose_xyz, res, xyz_res;
    DevBuf check;  // checked builds: status word of the kernels' index checks
    DevBuf ref_xyz_in, ref_xyz_out, ref_res;                 // host-memory form of dock_refine
    void* stage = nullptr;                                   // pinned staging of ligand uploads
    size_t stage_bytes = 0;
    std::map<std::string, std::unique_ptr<DevBuf>> pocket_sets;  // device pocket arrays per pocket list
    std::map<std::string, std::unique_ptr<Plan>> plans;
    dock_stats stats{};
    WorkTally tally;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the sweep kernel(s) of the last run
    bool timed = false;
    DbSlot db[2];                     // database pipeline stages
    cudaStream_t copy = nullptr;      // its uploads (non-blocking)
    ~dock_ctx() {
        plans.clear();
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (stage) cudaFreeHost(stage);
        if (copy) cudaStreamDestroy(copy);
    }
};

namespace {

int fail(dock_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

// A failed runtime call returns its code as DOCK_ERR_OUT_OF_MEMORY or DOCK_ERR_CUDA. The runtime's
// last-error state is cleared on the way out, so that a failure that leaves the context usable (an
// allocation that did not fit) is not reported again by the next call's launch checks.
#define CK(call)                                                                                           \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess) {                                                                           \
            (void)cudaGetLastError();                                                                      \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? DOCK_ERR_OUT_OF_MEMORY : DOCK_ERR_CUDA,     \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);              \
        }                                                                                                  \
    } while (0)

// Checked builds (GEODOCK_CHECKED): the device status word of the kernels' index checks, allocated on
// first use; other builds have none (NULL).
unsigned long long* check_word(dock_ctx* ctx) {
#ifdef GEODOCK_CHECKED
    if (!ctx->check.p && ctx->check.ensure(sizeof(unsigned long long)) == cudaSuccess)
        cudaMemset(ctx->check.p, 0, sizeof(unsigned long long));
    return ctx->check.as<unsigned long long>();
#else
    (void)ctx;
    return nullptr;
#endif
}

// Checked builds: wait for the work on stream s, read and clear the status word, and report a failed check
// as DOCK_ERR_CUDA with its code and index. Other builds return DOCK_OK at once.
int read_check(dock_ctx* ctx, cudaStream_t s, unsigned long long* word = nullptr) {
#ifdef GEODOCK_CHECKED
    unsigned long long* w = word ? word : check_word(ctx);
    if (!w) return fail(ctx, DOCK_ERR_OUT_OF_MEMORY, "checked build: no status word");
    unsigned long long v = 0;
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpy(&v, w, sizeof v, cudaMemcpyDeviceToHost));
    if (v) {
        CK(cudaMemset(w, 0, sizeof v));
        return fail(ctx, DOCK_ERR_CUDA, "index check %u failed at index %u (checked build)", (unsigned)(v >> 32),
                    (unsigned)(v & 0xffffffffu));
    }
#else
    (void)ctx;
    (void)s;
    (void)word;
#endif
    return DOCK_OK;
}

int n_angles(double step) {
    int P = (int)std::ceil(360.0 / step);
    while (P > 1 && (P - 1) * step >= 360.0) --P;
    while (P * step < 360.0) ++P;
    return P;
}

// Tile of tile peeling (Eq. 3 reading): the divisor of 360 that is a multiple
// of the step and lies nearest to sqrt(360 step); ties to the smaller one.
int peel_tile(double step) {
    double target = std::sqrt(360.0 * step);
    int best = -1;
    double bestd = 1e300;
    for (int x = 1; x <= 360; ++x) {
        if (360 % x) continue;
        double q = x / step;
        if (std::fabs(q - std::round(q)) > 1e-9 || q < 1.0 - 1e-9) continue;
        double d = std::fabs(x - target);
        if (d < bestd - 1e-12) {
            bestd = d;
            best = x;
        }
    }
    return best;
}

// Angle counts of a run's knobs, computed once per call (peel_tile searches the divisors of 360, too slow
// to repeat per ligand and sweep descriptor on large batches).
struct Steps {
    int P_hp = 1, P_lp = 1;
    int tile = 0;  // tile of tile peeling, 0 without it
};
Steps steps_of(const dock_knobs* k) {
    Steps s;
    s.P_hp = n_angles(k->hp_step);
    s.P_lp = n_angles(k->lp_step);
    if (k->enable_refinement) s.tile = peel_tile(k->hp_step);
    return s;
}

std::vector<float2> angle_table(const std::vector<double>& deg) {
    std::vector<float2> t(deg.size());
    const double rad = 3.14159265358979323846 / 180.0;
    for (size_t i = 0; i < deg.size(); ++i) t[i] = make_float2((float)std::cos(deg[i] * rad), (float)std::sin(deg[i] * rad));
    return t;
}

int check_knobs(dock_ctx* ctx, const dock_knobs* k) {
    if (!k) return fail(ctx, DOCK_ERR_INVALID_ARG, "knobs: NULL");
    if (!(k->hp_step >= 1.0 && k->hp_step <= 360.0) || !(k->lp_step >= 1.0 && k->lp_step <= 360.0))
        return fail(ctx, DOCK_ERR_INVALID_ARG, "knobs: steps must lie in [1, 360] degrees");
    if (k->repetitions < 0 || k->repetitions > 1000) return fail(ctx, DOCK_ERR_INVALID_ARG, "knobs: repetitions");
    if (k->n_poses < 1 || k->n_poses > DOCK_MAX_POSES) return fail(ctx, DOCK_ERR_INVALID_ARG, "knobs: n_poses");
    if (!(k->bump_thr >= 0.0) || !std::isfinite(k->bump_thr)) return fail(ctx, DOCK_ERR_INVALID_ARG, "knobs: bump_thr");
    if (!std::isfinite(k->threshold)) return fail(ctx, DOCK_ERR_INVALID_ARG, "knobs: threshold");
    if (k->score_mode < 0 || k->score_mode > 2) return fail(ctx, DOCK_ERR_INVALID_ARG, "knobs: score_mode");
    if (k->refine_steps < 0 || k->refine_steps > 1000) return fail(ctx, DOCK_ERR_INVALID_ARG, "knobs: refine_steps");
    if (k->enable_refinement && peel_tile(k->hp_step) < 0)
        return fail(ctx, DOCK_ERR_UNSUPPORTED, "knobs: no tile size divides 360 for this step");
    return DOCK_OK;
}

int trace_pmax(const dock_knobs* k) {
    int p = std::max(n_angles(k->hp_step), n_angles(k->lp_step));
    if (k->enable_refinement) {
        int x = peel_tile(k->hp_step);
        p = std::max(p, 1 + 360 / x + (int)std::lround(x / k->hp_step));
    }
    return p;
}

// Default tile shape. Two lanes share a pose (splitting its atoms) when the run
// has at least 16 poses, more for fewer poses, so that a warp holds no more
// poses than the run has; larger ligands get more lanes per pose (see
// lanes_log2). Up to 18 angles per chunk keep a thread within 128 registers,
// so two CTAs of 8 warps fit an SM; with one moving atom per pass the hot
// code stays small enough for the instruction cache at that occupancy.
dock_tile default_tile(const dock_knobs* k) {
    dock_tile t;
    int N = k->n_poses;
    t.lanes_per_pose = N >= 16 ? 2 : (N >= 8 ? 4 : 8);
    int ncand = n_angles(k->hp_step) - 1;
    t.angles_per_chunk = ncand <= 8 ? 8 : (ncand <= 12 ? 12 : 18);
    t.warps_per_cta = 8;
    if (k->score_mode == 2) {
        t.angles_per_chunk = 12;  // the only instantiation of the exact score
        t.warps_per_cta = 4;
    }
    return t;
}

// Shared-memory floats per warp for its poses' coordinates: 32 atoms of
// 32 / lanes_per_pose poses (never more than the batch needs), and at least
// one pose of the batch's largest ligand (which then runs one pose per warp).
int slice_floats(const dock_tile& t, int lmax) {
    const int base = (32 / t.lanes_per_pose) * std::min(32, lmax) * 3;
    return (std::max(base, 3 * lmax) + 3) & ~3;  // 16-byte multiple
}

// log2 of the lanes per pose for a ligand of l atoms: the smallest Q >= the
// tile's lanes_per_pose with (32/Q) poses x l atoms inside the warp's slice.
int lanes_log2(const dock_tile& t, int slice, int l) {
    int lq = 0;
    while ((1 << lq) < t.lanes_per_pose) ++lq;
    while (lq < 5 && (32 >> lq) * l * 3 > slice) ++lq;
    return lq;
}

// Shared memory of a CTA: per warp the coordinate slice, the bump list and
// the chunk's angle table.
size_t cta_smem(const dock_tile& t, int slice, int bw) {
    return (size_t)t.warps_per_cta * (slice + warp_extra_floats(t.angles_per_chunk, bw)) * sizeof(float);
}

// 64-bit bump words per lane: the largest phase of a sweep (flat hp or lp
// sweep, tile centres, or one tile's angles) in 64-candidate words.
int bump_words(const dock_knobs* k) {
    // with tile peeling a high-precision fragment sweeps the tile centres, then one tile: never the flat hp
    // candidates
    int m = n_angles(k->lp_step) - 1;
    if (k->enable_refinement) {
        int x = peel_tile(k->hp_step);
        m = std::max(m, std::max(360 / x, (int)std::lround(x / k->hp_step)));
    } else {
        m = std::max(m, n_angles(k->hp_step) - 1);
    }
    return std::max(1, (m + 63) / 64);
}

cudaError_t launch_sweep(int kc, const SweepParams& P, int mode, int clip, int grid, int block, size_t smem,
                         cudaStream_t s) {
    switch (kc) {
        case 8: return launch_sweep_kc8(P, mode, clip, grid, block, smem, s);
        case 12: return launch_sweep_kc12(P, mode, clip, grid, block, smem, s);
        case 18: return launch_sweep_kc18(P, mode, clip, grid, block, smem, s);
        default: return launch_sweep_kc36(P, mode, clip, grid, block, smem, s);
    }
}
cudaError_t occupancy(int kc, int mode, int clip, int block, size_t smem, int* n) {
    switch (kc) {
        case 8: return occupancy_kc8(mode, clip, block, smem, n);
        case 12: return occupancy_kc12(mode, clip, block, smem, n);
        case 18: return occupancy_kc18(mode, clip, block, smem, n);
        default: return occupancy_kc36(mode, clip, block, smem, n);
    }
}

std::string plan_key(int batch_id, const int32_t* pids, int np, const dock_knobs* k, const dock_tile& t, int plain) {
    char buf[512];
    snprintf(buf, sizeof buf, "%d|%a|%a|%a|%d|%d|%d|%d|%a|%d|%llu|%d|%d|%d|%d|", batch_id, k->hp_step, k->lp_step,
             k->threshold, k->repetitions, k->n_poses, k->enable_refinement, k->clip_box, k->bump_thr, k->score_mode,
             (unsigned long long)k->seed, t.lanes_per_pose, t.angles_per_chunk, t.warps_per_cta, plain);
    std::string s = buf;
    for (int i = 0; i < np; ++i) s += std::to_string(pids[i]) + ",";
    return s;
}

// Estimated cost of one warp task (pose group) of ligand b: candidate
// evaluations times moving atoms, plus the bump partner scans per chunk.
double task_cost(const BatchH& B, int b, const dock_knobs* k, const Steps& st, int Q, int kc) {
    double c = 0;
    for (int s = 0; s < B.nside[b]; ++s) {
        int si = B.side_off[b] + s;
        bool coarse = (double)B.side_m[si] / (double)B.l[b] <= k->threshold;
        int ncand = coarse ? st.P_lp - 1 : st.P_hp - 1;
        if (st.tile && !coarse) ncand = 360 / st.tile + (int)std::lround(st.tile / k->hp_step);
        int chunks = (ncand + kc - 1) / kc;
        int nslot = (B.side_nmov[si] + Q - 1) / Q;
        c += (double)nslot * (chunks * (kc * 15.0 + 25.0) + B.side_nfixB[si] * 7.0) + 40.0 * B.l[b] / Q;
    }
    return c * std::max(k->repetitions, 1) + B.l[b] * 20.0 / Q;
}

// Host preparation of ligands [i0, i1) of a batch: topology checks, the two
// fragments of every rotatable bond (Alg. 1: the left one holds the bond's
// lower atom index) as per-sweep atom lists, the refinement torsions and the
// bump-pair rows. Offsets in the outputs are relative to this range.
struct PrepOut {
    std::vector<SideDev> sides;
    std::vector<uint8_t> idx;
    std::vector<RefTorDev> rtor;
    std::vector<uint32_t> check;
    std::vector<int> side_m, side_nmov, side_nfixB;
    int err = 0;
    std::string msg;
};

void prep_range(const dock_ligand_batch* b, int i0, int i1, std::vector<LigDev>& lig, std::vector<RefLigDev>& rlig,
                PrepOut& out) {
    char buf[256];
    auto bad = [&](int code, const char* m) {
        out.err = code;
        out.msg = m;
    };
    // scratch reused across the range's ligands
    std::vector<int> deg, off, nbr, depth, queue, stack;
    std::vector<char> left;
    std::vector<uint32_t> lw, rw;
    std::vector<std::tuple<int, int, int>> tor_depth;  // (depth of c, torsion, moving side)
    for (int i = i0; i < i1; ++i) {
        const int a0 = b->atom_off[i], l = b->atom_off[i + 1] - a0;
        const int e0 = b->bond_off[i], ne = b->bond_off[i + 1] - e0;
        const int r0 = b->rot_off[i], nr = b->rot_off[i + 1] - r0;
        if (l < 1 || l > DOCK_MAX_ATOMS) {
            snprintf(buf, sizeof buf, "ligand %d: %d atoms", i, l);
            return bad(DOCK_ERR_INVALID_ARG, buf);
        }
        if (ne < 0 || nr < 0 || (ne > 0 && !b->bonds) || (nr > 0 && !b->rot)) {
            snprintf(buf, sizeof buf, "ligand %d: bad bond/rotamer offsets", i);
            return bad(DOCK_ERR_INVALID_ARG, buf);
        }
        // adjacency in CSR form
        deg.assign(l + 1, 0);
        for (int e = 0; e < ne; ++e) {
            const int u = b->bonds[2 * (e0 + e)], v = b->bonds[2 * (e0 + e) + 1];
            if (u < 0 || v < 0 || u >= l || v >= l || u == v) {
                snprintf(buf, sizeof buf, "ligand %d: bond %d has bad atoms", i, e);
                return bad(DOCK_ERR_INVALID_ARG, buf);
            }
            ++deg[u];
            ++deg[v];
        }
        off.assign(l + 1, 0);
        for (int a = 0; a < l; ++a) off[a + 1] = off[a] + deg[a];
        nbr.resize(2 * ne);
        for (int a = 0; a < l; ++a) deg[a] = off[a];
        for (int e = 0; e < ne; ++e) {
            const int u = b->bonds[2 * (e0 + e)], v = b->bonds[2 * (e0 + e) + 1];
            nbr[deg[u]++] = v;
            nbr[deg[v]++] = u;
        }
        double g[3] = {0, 0, 0};
        for (int a = 0; a < l; ++a)
            for (int d = 0; d < 3; ++d) {
                const float x = b->xyz[3 * (a0 + a) + d];
                if (!std::isfinite(x) || std::fabs(x) > 1e5f) {
                    snprintf(buf, sizeof buf, "ligand %d: coordinate out of range", i);
                    return bad(DOCK_ERR_INVALID_ARG, buf);
                }
                g[d] += (double)x;
            }
        LigDev& L = lig[i];
        L.atom_off = a0;
        L.l = l;
        L.nside = 2 * nr;
        L.side_off = (int)out.sides.size();
        for (int d = 0; d < 3; ++d) L.g[d] = g[d] / l;
        L.id = b->ids ? b->ids[i] : b->id_base + i;
        // graph depth from atom 0 (refinement order)
        depth.assign(l, -1);
        queue.assign(1, 0);
        depth[0] = 0;
        for (size_t h = 0; h < queue.size(); ++h)
            for (int k = off[queue[h]]; k < off[queue[h] + 1]; ++k)
                if (depth[nbr[k]] < 0) {
                    depth[nbr[k]] = depth[queue[h]] + 1;
                    queue.push_back(nbr[k]);
                }
        const int wpr = (l + 31) / 32;
        RefLigDev& RL = rlig[i];
        RL.tor_off = (int)out.rtor.size();
        RL.T = nr;
        RL.check_off = (int)out.check.size();
        RL.wpr = wpr;
        out.check.resize(out.check.size() + (size_t)l * wpr, 0u);
        tor_depth.clear();
        for (int r = 0; r < nr; ++r) {
            const int e = b->rot[r0 + r];
            if (e < 0 || e >= ne) {
                snprintf(buf, sizeof buf, "ligand %d: rotatable bond index %d", i, e);
                return bad(DOCK_ERR_INVALID_ARG, buf);
            }
            int u = b->bonds[2 * (e0 + e)], v = b->bonds[2 * (e0 + e) + 1];
            if (u > v) std::swap(u, v);
            // left fragment: atoms reachable from u without crossing (u, v)
            left.assign(l, 0);
            stack.assign(1, u);
            left[u] = 1;
            while (!stack.empty()) {
                const int x = stack.back();
                stack.pop_back();
                for (int k = off[x]; k < off[x + 1]; ++k) {
                    const int y = nbr[k];
                    if ((x == u && y == v) || (x == v && y == u)) continue;
                    if (!left[y]) {
                        left[y] = 1;
                        stack.push_back(y);
                    }
                }
            }
            if (left[v]) {
                snprintf(buf, sizeof buf, "ligand %d: rotatable bond %d lies on a ring", i, e);
                return bad(DOCK_ERR_TOPOLOGY, buf);
            }
            // refinement torsion: the side without atom 0 moves (side 1 = right fragment when atom 0 is left)
            tor_depth.emplace_back(depth[left[0] ? v : u], r, left[0] ? 1 : 0);
            // bump-pair rows: every pair this torsion moves
            lw.assign(wpr, 0u);
            rw.assign(wpr, 0u);
            for (int a = 0; a < l; ++a) {
                if (left[a] && a != u) lw[a >> 5] |= 1u << (a & 31);
                if (!left[a] && a != v) rw[a >> 5] |= 1u << (a & 31);
            }
            uint32_t* rows = out.check.data() + RL.check_off;
            for (int a = 0; a < l; ++a) {
                const std::vector<uint32_t>* other = (lw[a >> 5] >> (a & 31)) & 1u   ? &rw
                                                     : (rw[a >> 5] >> (a & 31)) & 1u ? &lw
                                                                                      : nullptr;
                if (other)
                    for (int w = 0; w < wpr; ++w) rows[(size_t)a * wpr + w] |= (*other)[w];
            }
            for (int side = 0; side < 2; ++side) {
                // side 0: the left fragment moves (c = u, b = v); side 1: the right one (c = v, b = u)
                const int c = side == 0 ? u : v, bb = side == 0 ? v : u;
                SideDev sd{};
                sd.c = (uint8_t)c;
                sd.b = (uint8_t)bb;
                sd.mov_off = (int)out.idx.size();
                int m = 0;
                for (int a = 0; a < l; ++a) {
                    const bool moving = side == 0 ? left[a] != 0 : left[a] == 0;
                    if (!moving) continue;
                    ++m;
                    if (a != c) out.idx.push_back((uint8_t)a);
                }
                sd.m = (uint8_t)m;
                sd.nmov = (uint8_t)(m - 1);
                sd.fix_off = (int)out.idx.size();
                for (int a = 0; a < l; ++a) {
                    const bool moving = side == 0 ? left[a] != 0 : left[a] == 0;
                    if (!moving && a != bb) out.idx.push_back((uint8_t)a);
                }
                out.idx.push_back((uint8_t)bb);
                out.idx.push_back((uint8_t)c);
                sd.nfixB = (uint8_t)(l - m - 1);
                sd.nfixS = (uint8_t)(l - m + 1);
                out.sides.push_back(sd);
                out.side_m.push_back(m);
                out.side_nmov.push_back(m - 1);
                out.side_nfixB.push_back(l - m - 1);
            }
        }
        // deepest bond first, ties in bond order
        std::stable_sort(tor_depth.begin(), tor_depth.end(),
                         [](const std::tuple<int, int, int>& x, const std::tuple<int, int, int>& y) {
                             return std::get<0>(x) > std::get<0>(y);
                         });
        for (const auto& td : tor_depth) out.rtor.push_back({2 * std::get<1>(td) + std::get<2>(td), std::get<1>(td)});
    }
}

}  // namespace

// ======================================================================== API

extern "C" {

int dock_create(dock_ctx** out, int device) {
    if (!out) return DOCK_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return DOCK_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return DOCK_ERR_CUDA;
    dock_ctx* c = new dock_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) {
        delete c;
        return DOCK_ERR_CUDA;
    }
    *out = c;
    return DOCK_OK;
}

void dock_destroy(dock_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    delete ctx;
}

const char* dock_last_error(const dock_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int dock_init_pocket(dock_ctx* ctx, const dock_pocket* p, int* pocket_id) {
    Range range("dock_init_pocket");
    if (!ctx || !p || !pocket_id) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_init_pocket: NULL argument");
    CK(cudaSetDevice(ctx->device));
    if (p->nx < 2 || p->ny < 2 || p->nz < 2 || p->nx > DOCK_MAX_GRID || p->ny > DOCK_MAX_GRID || p->nz > DOCK_MAX_GRID)
        return fail(ctx, DOCK_ERR_INVALID_ARG, "pocket: grid size out of range");
    if (!(p->h > 0.0) || !std::isfinite(p->h)) return fail(ctx, DOCK_ERR_INVALID_ARG, "pocket: h must be > 0");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(p->origin[a]) || !std::isfinite(p->centre[a]))
            return fail(ctx, DOCK_ERR_INVALID_ARG, "pocket: non-finite origin/centre");
    int64_t nv = (int64_t)p->nx * p->ny * p->nz;
    // the largest squared distance between voxels must fit the 16-bit field
    int64_t dmax = (int64_t)(p->nx - 1) * (p->nx - 1) + (int64_t)(p->ny - 1) * (p->ny - 1) + (int64_t)(p->nz - 1) * (p->nz - 1);
    PocketH ph;
    ph.K.reset(new DevBuf());
    CK(ph.K->ensure(nv * sizeof(uint16_t)));
    if (p->K) {
        for (int64_t v = 0; v < nv; ++v)
            if (p->K[v] < 1) return fail(ctx, DOCK_ERR_INVALID_ARG, "pocket: field values must be >= 1");
        CK(cudaMemcpy(ph.K->p, p->K, nv * sizeof(uint16_t), cudaMemcpyHostToDevice));
    } else {
        if (!p->pts || p->npts < 1) return fail(ctx, DOCK_ERR_INVALID_ARG, "pocket: no probe points");
        if (dmax > 65535) return fail(ctx, DOCK_ERR_INVALID_ARG, "pocket: grid too large for 16-bit distances");
        std::vector<int4> pts(p->npts);
        for (int j = 0; j < p->npts; ++j) {
            int x = p->pts[3 * j], y = p->pts[3 * j + 1], z = p->pts[3 * j + 2];
            if (x < 0 || y < 0 || z < 0 || x >= p->nx || y >= p->ny || z >= p->nz)
                return fail(ctx, DOCK_ERR_INVALID_ARG, "pocket: probe point %d outside the grid", j);
            pts[j] = make_int4(x, y, z, 0);
        }
        DevBuf dp;
        CK(dp.ensure(pts.size() * sizeof(int4)));
        CK(cudaMemcpy(dp.p, pts.data(), pts.size() * sizeof(int4), cudaMemcpyHostToDevice));
        int threads = 256;
        int64_t blocks = (nv + threads - 1) / threads;
        field_kernel<<<(unsigned)blocks, threads>>>(ph.K->as<uint16_t>(), p->nx, p->ny, p->nz, dp.as<int4>(), p->npts);
        CK(cudaGetLastError());
        CK(cudaDeviceSynchronize());
    }
    // padded 32-bit copy for the sweep's unchecked lookups, held as a texture: point sampling at
    // unnormalized coordinates returns the voxel at the floor of each coordinate, from a
    // cache-friendly 3D layout; the linear copy is only the array's source
    {
        const int64_t np = (int64_t)(p->nx + 2 * PAD) * (p->ny + 2 * PAD) * (p->nz + 2 * PAD);
        DevBuf lin;
        CK(lin.ensure(np * sizeof(uint32_t)));
        pad_field_kernel<<<(unsigned)((np + 255) / 256), 256>>>(lin.as<uint32_t>(), ph.K->as<uint16_t>(), p->nx,
                                                                p->ny, p->nz);
        CK(cudaGetLastError());
        CK(cudaDeviceSynchronize());
        const size_t ex = (size_t)(p->nx + 2 * PAD), ey = (size_t)(p->ny + 2 * PAD), ez = (size_t)(p->nz + 2 * PAD);
        ph.Kt.reset(new FieldTex());
        cudaChannelFormatDesc fd = cudaCreateChannelDesc<unsigned>();
        CK(cudaMalloc3DArray(&ph.Kt->arr, &fd, make_cudaExtent(ex, ey, ez)));
        cudaMemcpy3DParms cp = {};
        cp.srcPtr = make_cudaPitchedPtr(lin.p, ex * sizeof(uint32_t), ex, ey);
        cp.dstArray = ph.Kt->arr;
        cp.extent = make_cudaExtent(ex, ey, ez);
        cp.kind = cudaMemcpyDeviceToDevice;
        CK(cudaMemcpy3D(&cp));
        cudaResourceDesc rd = {};
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = ph.Kt->arr;
        cudaTextureDesc td = {};
        td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        CK(cudaCreateTextureObject(&ph.Kt->tex, &rd, &td, nullptr));
        CK(cudaDeviceSynchronize());  // before the linear copy is freed
    }
    // the 2x2x2 corners of every voxel, one 16-byte texel each, for the trilinear score
    {
        DevBuf lin;
        CK(lin.ensure(nv * sizeof(uint4)));
        corner_field_kernel<<<(unsigned)((nv + 255) / 256), 256>>>(lin.as<uint4>(), ph.K->as<uint16_t>(), p->nx, p->ny,
                                                                   p->nz);
        CK(cudaGetLastError());
        CK(cudaDeviceSynchronize());
        ph.Kc.reset(new FieldTex());
        cudaChannelFormatDesc fd = cudaCreateChannelDesc<uint4>();
        CK(cudaMalloc3DArray(&ph.Kc->arr, &fd, make_cudaExtent(p->nx, p->ny, p->nz)));
        cudaMemcpy3DParms cp = {};
        cp.srcPtr = make_cudaPitchedPtr(lin.p, (size_t)p->nx * sizeof(uint4), p->nx, p->ny);
        cp.dstArray = ph.Kc->arr;
        cp.extent = make_cudaExtent(p->nx, p->ny, p->nz);
        cp.kind = cudaMemcpyDeviceToDevice;
        CK(cudaMemcpy3D(&cp));
        cudaResourceDesc rd = {};
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = ph.Kc->arr;
        cudaTextureDesc td = {};
        td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        CK(cudaCreateTextureObject(&ph.Kc->tex, &rd, &td, nullptr));
        CK(cudaDeviceSynchronize());  // before the linear copy is freed
    }
    // probe points for the exact score (Eq. 1's inner minimum without the grid)
    if (p->pts && p->npts > 0) {
        std::vector<float4> q(p->npts);
        for (int j = 0; j < p->npts; ++j) {
            int x = p->pts[3 * j], y = p->pts[3 * j + 1], z = p->pts[3 * j + 2];
            if (x < 0 || y < 0 || z < 0 || x >= p->nx || y >= p->ny || z >= p->nz)
                return fail(ctx, DOCK_ERR_INVALID_ARG, "pocket: probe point %d outside the grid", j);
            q[j] = make_float4(x + 0.5f, y + 0.5f, z + 0.5f, 0.f);
        }
        ph.pts.reset(new DevBuf());
        CK(ph.pts->ensure(q.size() * sizeof(float4)));
        CK(cudaMemcpy(ph.pts->p, q.data(), q.size() * sizeof(float4), cudaMemcpyHostToDevice));
        ph.d.pts = ph.pts->as<float4>();
        ph.d.npts = p->npts;
    }
    ph.d.K = ph.K->as<uint16_t>();
    ph.d.Kt = ph.Kt->tex;
    ph.d.Kc = ph.Kc->tex;
    ph.d.nx = p->nx;
    ph.d.ny = p->ny;
    ph.d.nz = p->nz;
    ph.d.h = p->h;
    for (int a = 0; a < 3; ++a) {
        ph.d.origin[a] = p->origin[a];
        ph.d.centre[a] = p->centre[a];
    }
    ph.dev.reset(new DevBuf());
    CK(ph.dev->ensure(sizeof(PocketDev)));
    CK(cudaMemcpy(ph.dev->p, &ph.d, sizeof(PocketDev), cudaMemcpyHostToDevice));
    ph.live = true;
    ctx->pockets.push_back(std::move(ph));
    *pocket_id = (int)ctx->pockets.size() - 1;
    return DOCK_OK;
}

int dock_pocket_field(dock_ctx* ctx, int pocket_id, uint16_t* K) {
    if (!ctx || !K || pocket_id < 0 || pocket_id >= (int)ctx->pockets.size() || !ctx->pockets[pocket_id].live)
        return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_pocket_field: bad arguments");
    CK(cudaSetDevice(ctx->device));
    const PocketDev& d = ctx->pockets[pocket_id].d;
    CK(cudaMemcpy(K, d.K, (size_t)d.nx * d.ny * d.nz * sizeof(uint16_t), cudaMemcpyDeviceToHost));
    return DOCK_OK;
}

}  // extern "C"

namespace {

// Validate a batch and prepare it on the host (Alg. 1's fragment lists per
// rotatable bond, refinement torsions, bump-pair rows); fills B's host fields.
int prep_batch(dock_ctx* ctx, const dock_ligand_batch* b, BatchH& B, BatchImage& im) {
    if (b->n < 0) return fail(ctx, DOCK_ERR_INVALID_ARG, "batch: n < 0");
    if (b->n > 0 && (!b->atom_off || !b->xyz || !b->bond_off || !b->rot_off))
        return fail(ctx, DOCK_ERR_INVALID_ARG, "batch: NULL array");
    if (b->n > 0 && (b->atom_off[0] != 0 || b->bond_off[0] != 0 || b->rot_off[0] != 0))
        return fail(ctx, DOCK_ERR_INVALID_ARG, "batch: offsets must start at 0");
    const int n = b->n;
    B = BatchH();
    B.n = n;
    std::vector<LigDev>& lig = im.lig;
    std::vector<RefLigDev>& rlig = im.rlig;
    lig.assign(n, LigDev{});
    rlig.assign(n, RefLigDev{});
    // the ligands are independent: ranges of them are prepared in parallel, then joined in order
    const int hw = std::max(1, (int)std::thread::hardware_concurrency());
    const int nt = std::max(1, std::min(hw, n / 64));
    std::vector<PrepOut> parts(nt);
    std::vector<std::thread> pool;
    for (int t = 0; t < nt; ++t) {
        const int i0 = (int)((int64_t)n * t / nt), i1 = (int)((int64_t)n * (t + 1) / nt);
        if (t + 1 < nt)
            pool.emplace_back([&, t, i0, i1]() { prep_range(b, i0, i1, lig, rlig, parts[t]); });
        else
            prep_range(b, i0, i1, lig, rlig, parts[t]);
    }
    for (auto& th : pool) th.join();
    for (const PrepOut& o : parts)
        if (o.err) return fail(ctx, o.err, "%s", o.msg.c_str());
    size_t nside = 0, nidx = 0, ntor = 0, nchk = 0;
    for (const PrepOut& o : parts) {
        nside += o.sides.size();
        nidx += o.idx.size();
        ntor += o.rtor.size();
        nchk += o.check.size();
    }
    std::vector<SideDev>& sides = im.sides;
    std::vector<uint8_t>& idx = im.idx;
    std::vector<RefTorDev>& rtor = im.rtor;
    std::vector<uint32_t>& check = im.check;
    sides.clear();
    idx.clear();
    rtor.clear();
    check.clear();
    sides.reserve(nside);
    idx.reserve(nidx);
    rtor.reserve(ntor);
    check.reserve(nchk);
    for (int t = 0; t < nt; ++t) {
        const PrepOut& o = parts[t];
        const int i0 = (int)((int64_t)n * t / nt), i1 = (int)((int64_t)n * (t + 1) / nt);
        const int sb = (int)sides.size(), ib = (int)idx.size(), tb = (int)rtor.size(), cb = (int)check.size();
        for (int i = i0; i < i1; ++i) {
            lig[i].side_off += sb;
            rlig[i].tor_off += tb;
            rlig[i].check_off += cb;
        }
        for (SideDev sd : o.sides) {
            sd.mov_off += ib;
            sd.fix_off += ib;
            sides.push_back(sd);
        }
        idx.insert(idx.end(), o.idx.begin(), o.idx.end());
        rtor.insert(rtor.end(), o.rtor.begin(), o.rtor.end());  // sides index the ligand's own
        check.insert(check.end(), o.check.begin(), o.check.end());
        B.side_m.insert(B.side_m.end(), o.side_m.begin(), o.side_m.end());
        B.side_nmov.insert(B.side_nmov.end(), o.side_nmov.begin(), o.side_nmov.end());
        B.side_nfixB.insert(B.side_nfixB.end(), o.side_nfixB.begin(), o.side_nfixB.end());
    }
    for (int i = 0; i < n; ++i) {
        B.l.push_back(lig[i].l);
        B.nside.push_back(lig[i].nside);
        B.side_off.push_back(lig[i].side_off);
        B.atom_off.push_back(lig[i].atom_off);
        B.lmax = std::max(B.lmax, lig[i].l);
        B.tmax = std::max(B.tmax, rlig[i].T);
    }
    B.natoms = n > 0 ? b->atom_off[n] : 0;
    B.nside_total = (int)sides.size();
    B.nidx = (int)idx.size();
    B.ntor = (int)rtor.size();
    B.nchk = (int)check.size();
    // one device allocation, 256-byte aligned parts
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    im.xyz = b->xyz;
    im.o_lig = 0;
    im.o_side = al(im.o_lig + lig.size() * sizeof(LigDev));
    im.o_idx = al(im.o_side + sides.size() * sizeof(SideDev));
    im.o_xyz = al(im.o_idx + idx.size());
    im.o_rlig = al(im.o_xyz + (size_t)B.natoms * 3 * sizeof(float));
    im.o_rtor = al(im.o_rlig + rlig.size() * sizeof(RefLigDev));
    im.o_chk = al(im.o_rtor + rtor.size() * sizeof(RefTorDev));
    im.total = al(im.o_chk + check.size() * sizeof(uint32_t)) + 256;
    return DOCK_OK;
}

// Write a prepared batch into host memory h (im.total bytes) in its device layout.
void stage_batch(const BatchImage& im, int natoms, uint8_t* h) {
    std::memcpy(h + im.o_lig, im.lig.data(), im.lig.size() * sizeof(LigDev));
    std::memcpy(h + im.o_side, im.sides.data(), im.sides.size() * sizeof(SideDev));
    std::memcpy(h + im.o_idx, im.idx.data(), im.idx.size());
    if (natoms) std::memcpy(h + im.o_xyz, im.xyz, (size_t)natoms * 3 * sizeof(float));
    std::memcpy(h + im.o_rlig, im.rlig.data(), im.rlig.size() * sizeof(RefLigDev));
    std::memcpy(h + im.o_rtor, im.rtor.data(), im.rtor.size() * sizeof(RefTorDev));
    std::memcpy(h + im.o_chk, im.check.data(), im.check.size() * sizeof(uint32_t));
}

// Point B's device arrays into the allocation d holding the staged image.
void bind_batch(BatchH& B, const BatchImage& im, uint8_t* d) {
    B.d_lig = reinterpret_cast<LigDev*>(d + im.o_lig);
    B.d_side = reinterpret_cast<SideDev*>(d + im.o_side);
    B.d_idx = d + im.o_idx;
    B.d_xyz0 = reinterpret_cast<float*>(d + im.o_xyz);
    B.d_rlig = reinterpret_cast<RefLigDev*>(d + im.o_rlig);
    B.d_rtor = reinterpret_cast<RefTorDev*>(d + im.o_rtor);
    B.d_check = reinterpret_cast<uint32_t*>(d + im.o_chk);
}

// Pinned host memory that grows on demand.
int ensure_pinned(dock_ctx* ctx, void** p, size_t* have, size_t want) {
    if (*have >= want && *p) return DOCK_OK;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *have = 0;
    CK(cudaHostAlloc(p, want, cudaHostAllocDefault));
    *have = want;
    return DOCK_OK;
}

}  // namespace

extern "C" {

int dock_upload_ligands(dock_ctx* ctx, const dock_ligand_batch* b, int* batch_id) {
    Range range("dock_upload_ligands");
    if (!ctx || !b || !batch_id) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_upload_ligands: NULL argument");
    CK(cudaSetDevice(ctx->device));
    BatchH B;
    BatchImage im;
    int rc = prep_batch(ctx, b, B, im);
    if (rc) return rc;
    // one device allocation and one copy from a pinned staging buffer
    if ((rc = ensure_pinned(ctx, &ctx->stage, &ctx->stage_bytes, im.total))) return rc;
    uint8_t* h = static_cast<uint8_t*>(ctx->stage);
    stage_batch(im, B.natoms, h);
    B.mem.reset(new DevBuf());
    CK(B.mem->ensure(im.total));
    CK(cudaMemcpy(B.mem->p, h, im.total, cudaMemcpyHostToDevice));
    bind_batch(B, im, B.mem->as<uint8_t>());
    B.live = true;
    ctx->batches.push_back(std::move(B));
    *batch_id = (int)ctx->batches.size() - 1;
    return DOCK_OK;
}

int dock_release_batch(dock_ctx* ctx, int batch_id) {
    if (!ctx || batch_id < 0 || batch_id >= (int)ctx->batches.size() || !ctx->batches[batch_id].live)
        return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_release_batch: bad batch");
    CK(cudaSetDevice(ctx->device));
    CK(cudaDeviceSynchronize());
    ctx->batches[batch_id] = BatchH();
    std::string pre = std::to_string(batch_id) + "|";
    for (auto it = ctx->plans.begin(); it != ctx->plans.end();)
        it = it->first.compare(0, pre.size(), pre) == 0 ? ctx->plans.erase(it) : std::next(it);
    return DOCK_OK;
}

int dock_trace_pmax(const dock_knobs* k) { return k ? trace_pmax(k) : -1; }

int dock_set_tile(dock_ctx* ctx, const dock_tile* t) {
    if (!ctx || !t) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_set_tile: NULL");
    if (t->lanes_per_pose && t->lanes_per_pose != 1 && t->lanes_per_pose != 2 && t->lanes_per_pose != 4 &&
        t->lanes_per_pose != 8)
        return fail(ctx, DOCK_ERR_INVALID_ARG, "tile: lanes_per_pose must be 1, 2, 4 or 8");
    if (t->angles_per_chunk && t->angles_per_chunk != 8 && t->angles_per_chunk != 12 && t->angles_per_chunk != 18 &&
        t->angles_per_chunk != 36)
        return fail(ctx, DOCK_ERR_INVALID_ARG, "tile: angles_per_chunk must be 8, 12, 18 or 36");
    if (t->warps_per_cta < 0 || t->warps_per_cta > 8) return fail(ctx, DOCK_ERR_INVALID_ARG, "tile: warps 1..8");
    ctx->tile = *t;
    return DOCK_OK;
}

int dock_get_tile(const dock_ctx* ctx, dock_tile* t) {
    if (!ctx || !t) return DOCK_ERR_INVALID_ARG;
    *t = ctx->tile;
    return DOCK_OK;
}

int dock_last_stats(const dock_ctx* ctx_, dock_stats* s) {
    if (!ctx_ || !s) return DOCK_ERR_INVALID_ARG;
    dock_ctx* ctx = const_cast<dock_ctx*>(ctx_);
    if (ctx->timed) {
        float ms = 0.f;
        CK(cudaEventSynchronize(ctx->ev1));
        CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
        ctx->stats.sweep_ms = ms;
        ctx->timed = false;
    }
    WorkTally& W = ctx->tally;
    if (W.pending && W.skipped && W.npairs > 0) {
        // repetitions left out at a fixed point were not computed: count only the work done
        std::vector<unsigned> sk(W.npairs);
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(sk.data(), W.skipped->p, (size_t)W.npairs * sizeof(unsigned), cudaMemcpyDeviceToHost));
        uint64_t reps = 0, c = 0, u = 0, bd = 0, pr = 0;
        for (int pair = 0; pair < W.npairs; ++pair) {
            const int b = pair % W.nlig;
            reps += sk[pair];
            c += sk[pair] * W.cand[b];
            u += sk[pair] * W.upd[b];
            bd += sk[pair] * W.bounds[b];
            pr += sk[pair] * W.pairs[b];
        }
        unsigned long long gated = 0;
        if (W.looked) CK(cudaMemcpy(&gated, W.looked->p, sizeof gated, cudaMemcpyDeviceToHost));
        ctx->stats.pose_reps_skipped = reps;
        ctx->stats.lookups_skipped = gated;
        ctx->stats.candidates -= c;
        ctx->stats.atom_updates -= u + gated;
        ctx->stats.pair_bounds -= bd;
        ctx->stats.bump_pairs -= pr;
        W.pending = false;
    }
    *s = ctx->stats;
    return DOCK_OK;
}

}  // extern "C"

namespace {

// Resolve the tile shape: forced fields, else the autotuned shape for this
// (batch, knobs), else the default.
dock_tile resolve_tile(dock_ctx* ctx, int batch_id, const dock_knobs* k) {
    dock_tile t = default_tile(k);
    auto it = ctx->tuned.find(plan_key(batch_id, nullptr, 0, k, dock_tile{0, 0, 0}, 0));
    if (it != ctx->tuned.end()) t = it->second;
    if (ctx->tile.lanes_per_pose) t.lanes_per_pose = ctx->tile.lanes_per_pose;
    if (ctx->tile.angles_per_chunk) t.angles_per_chunk = ctx->tile.angles_per_chunk;
    if (ctx->tile.warps_per_cta) t.warps_per_cta = ctx->tile.warps_per_cta;
    if (k->score_mode == 2) t.angles_per_chunk = 12;
    return t;
}

// Copy host data into buf (allocated, or grown, on demand). With a stream the
// copy is enqueued there (a pageable source is staged before the call returns).
int upload(dock_ctx* ctx, std::unique_ptr<DevBuf>& buf, const void* src, size_t bytes, cudaStream_t cs = nullptr) {
    if (!buf) buf.reset(new DevBuf());
    CK(buf->ensure(bytes));
    if (bytes) {
        if (cs) CK(cudaMemcpyAsync(buf->p, src, bytes, cudaMemcpyHostToDevice, cs));
        else CK(cudaMemcpy(buf->p, src, bytes, cudaMemcpyHostToDevice));
    }
    return DOCK_OK;
}

// The context's scratch (queue head, per-pose keys and coordinates, per-pair
// results) sized for a run of np pockets x nlig ligands (natoms atoms) x N
// poses. Growing it moves the buffers, so every cached plan (and its captured
// graph) is dropped.
int ensure_scratch(dock_ctx* ctx, int np, int nlig, int natoms, int N) {
    const int64_t npairs = (int64_t)np * nlig;
    const size_t need[5] = {sizeof(unsigned), (size_t)npairs * N * sizeof(unsigned long long),
                            (size_t)np * natoms * N * 3 * sizeof(float), (size_t)npairs * sizeof(dock_result),
                            (size_t)np * natoms * 3 * sizeof(float)};
    DevBuf* bufs[5] = {&ctx->counter, &ctx->pose_key, &ctx->pose_xyz, &ctx->res, &ctx->xyz_res};
    bool grow = false;
    for (int i = 0; i < 5; ++i) grow = grow || !bufs[i]->p || bufs[i]->n < need[i];
    if (grow) {
        CK(cudaDeviceSynchronize());
        ctx->plans.clear();
        for (int i = 0; i < 5; ++i) CK(bufs[i]->ensure(need[i]));
    }
    return DOCK_OK;
}

int build_plan(dock_ctx* ctx, const BatchH& B, const int32_t* pids, int np, const dock_knobs* k, const dock_tile& t,
               int plain, Plan* pl, cudaStream_t cs);

// Build (or fetch) the plan of a run: pockets, angle tables, tasks, launch shape.
int get_plan(dock_ctx* ctx, int batch_id, const int32_t* pids, int np, const dock_knobs* k, int plain, Plan** out) {
    const dock_tile t = resolve_tile(ctx, batch_id, k);
    // a forced lanes_per_pose also turns off the split of heavy ligands (build_plan), so it is part of the key
    const std::string key = plan_key(batch_id, pids, np, k, t, plain) + (ctx->tile.lanes_per_pose ? "forced" : "");
    auto it = ctx->plans.find(key);
    if (it != ctx->plans.end()) {
        *out = it->second.get();
        return DOCK_OK;
    }
    const BatchH& B = ctx->batches[batch_id];
    int rc = ensure_scratch(ctx, np, B.n, B.natoms, k->n_poses);
    if (rc) return rc;
    std::unique_ptr<Plan> pl(new Plan());
    if ((rc = build_plan(ctx, B, pids, np, k, t, plain, pl.get(), nullptr))) return rc;
    *out = pl.get();
    ctx->plans[key] = std::move(pl);
    return DOCK_OK;
}

// Fill a plan for batch B: pockets, angle tables, tasks, step choices, launch
// shape. Its buffers are reused when big enough; with a stream cs the uploads
// are enqueued there. The context's scratch must already fit the run.
int build_plan(dock_ctx* ctx, const BatchH& B, const int32_t* pids, int np, const dock_knobs* k, const dock_tile& t,
               int plain, Plan* pl, cudaStream_t cs) {
    pl->Q = t.lanes_per_pose;
    pl->kc = t.angles_per_chunk;
    pl->W = t.warps_per_cta;
    pl->block = 32 * pl->W;
    pl->slice = slice_floats(t, B.lmax);
    const int N = k->n_poses;
    pl->npairs = np * B.n;
    // pockets
    std::vector<PocketDev> pd(np);
    for (int i = 0; i < np; ++i) pd[i] = ctx->pockets[pids[i]].d;
    int rc = upload(ctx, pl->pockets, pd.data(), pd.size() * sizeof(PocketDev), cs);
    if (rc) return rc;
    // angle tables (host FP64 cos/sin rounded to FP32)
    const int P_hp = n_angles(k->hp_step), P_lp = n_angles(k->lp_step);
    std::vector<double> a_hp(P_hp), a_lp(P_lp), a_peel;
    for (int i = 0; i < P_hp; ++i) a_hp[i] = i * k->hp_step;
    for (int i = 0; i < P_lp; ++i) a_lp[i] = i * k->lp_step;
    int n_tiles = 0, per_tile = 0;
    if (k->enable_refinement) {
        int x = peel_tile(k->hp_step);
        n_tiles = 360 / x;
        per_tile = (int)std::lround(x / k->hp_step);
        for (int i = 0; i < n_tiles; ++i) a_peel.push_back(i * x + 0.5 * x);
    } else {
        a_peel.push_back(0.0);
    }
    if ((rc = upload(ctx, pl->cs_hp, angle_table(a_hp).data(), P_hp * sizeof(float2), cs))) return rc;
    if ((rc = upload(ctx, pl->cs_lp, angle_table(a_lp).data(), P_lp * sizeof(float2), cs))) return rc;
    if ((rc = upload(ctx, pl->cs_peel, angle_table(a_peel).data(), a_peel.size() * sizeof(float2), cs))) return rc;
    // tasks: (pair, pose group); batched form in descending cost (longest first),
    // plain form in pair order
    std::vector<int2> tasks;
    std::vector<double> cost;
    pl->task_off.assign(pl->npairs + 1, 0);
    const Steps st = steps_of(k);
    std::vector<int> lqs(B.n);
    std::vector<double> cb(B.n);
    for (int b = 0; b < B.n; ++b) {
        lqs[b] = lanes_log2(t, pl->slice, B.l[b]);
        cb[b] = task_cost(B, b, k, st, 1 << lqs[b], pl->kc);
    }
    // A launch lasts at least as long as its longest task. With the nearest-voxel score (exact integer
    // sums: results do not depend on the lanes a pose runs on), a ligand whose task would cost more than
    // 0.8 of the average load of a warp slot gets twice the lanes per pose (half the poses per task),
    // again while that holds: the heaviest ligands of a batch, or every ligand of a small batch. A
    // lanes_per_pose forced by dock_set_tile is kept as it is.
    if (!plain && k->score_mode == 0 && !ctx->tile.lanes_per_pose) {
        const double slots = (double)(pl->kc <= 18 ? 2 : 1) * ctx->num_sms * pl->W;
        for (int pass = 0; pass < 5; ++pass) {
            double work = 0;
            for (int b = 0; b < B.n; ++b) work += (double)np * ((N + (32 >> lqs[b]) - 1) / (32 >> lqs[b])) * cb[b];
            bool split = false;
            for (int b = 0; b < B.n; ++b)
                if (cb[b] > 0.8 * work / slots && lqs[b] < 5) {
                    ++lqs[b];
                    cb[b] = task_cost(B, b, k, st, 1 << lqs[b], pl->kc);
                    split = true;
                }
            if (!split) break;
        }
    }
    for (int pk = 0; pk < np; ++pk)
        for (int b = 0; b < B.n; ++b) {
            const int lq = lqs[b];
            const int G = 32 >> lq;
            const int ngroup = (N + G - 1) / G;
            const double c = cb[b];
            for (int g = 0; g < ngroup; ++g) {
                tasks.push_back(make_int2(pk * B.n + b, g | (lq << 16)));
                cost.push_back(c);
            }
            pl->task_off[pk * B.n + b + 1] = (int)tasks.size();
        }
    if (!plain) {
        std::vector<int> order(tasks.size());
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b2) { return cost[a] > cost[b2]; });
        std::vector<int2> sorted(tasks.size());
        for (size_t i = 0; i < order.size(); ++i) sorted[i] = tasks[order[i]];
        tasks.swap(sorted);
    }
    pl->ntask = (int)tasks.size();
    if ((rc = upload(ctx, pl->tasks, tasks.data(), tasks.size() * sizeof(int2), cs))) return rc;
    SweepParams& P = pl->P;
    P.lig = B.d_lig;
    P.side = B.d_side;
    P.idx = B.d_idx;
    P.xyz0 = B.d_xyz0;
    P.pockets = pl->pockets->as<PocketDev>();
    P.tasks = pl->tasks->as<int2>();
    P.ntask = pl->ntask;
    P.npockets = np;
    P.nidx = B.nidx;
    P.check = check_word(ctx);
    P.nlig = B.n;
    P.natoms = B.natoms;
    P.counter = ctx->counter.as<unsigned>();
    P.n_poses = N;
    P.repetitions = k->repetitions;
    P.slice = pl->slice;
    P.threshold = k->threshold;
    {
        // Alg. 2's step choice per sweep descriptor, decided once on the host
        std::vector<uint8_t> co(std::max(1, B.nside_total), 0);
        for (int b = 0; b < B.n; ++b)
            for (int si = 0; si < B.nside[b]; ++si) {
                const int g = B.side_off[b] + si;
                co[g] = (double)B.side_m[g] / (double)B.l[b] <= k->threshold ? 1 : 0;
            }
        if ((rc = upload(ctx, pl->coarse, co.data(), co.size(), cs))) return rc;
    }
    P.coarse = pl->coarse->as<uint8_t>();
    P.bump_thr = k->bump_thr;
    P.seed = k->seed;
    P.cs_hp = pl->cs_hp->as<float2>();
    P.cs_lp = pl->cs_lp->as<float2>();
    P.P_hp = P_hp;
    P.P_lp = P_lp;
    P.peel = k->enable_refinement ? 1 : 0;
    P.hp_step = (float)k->hp_step;
    P.lp_step = (float)k->lp_step;
    P.tile = k->enable_refinement ? (float)peel_tile(k->hp_step) : 0.f;
    P.cs_peel = pl->cs_peel->as<float2>();
    P.n_tiles = n_tiles;
    P.per_tile = per_tile;
    P.pose_key = ctx->pose_key.as<unsigned long long>();
    P.pose_xyz = ctx->pose_xyz.as<float>();
    if (!pl->skipped) pl->skipped.reset(new DevBuf());
    CK(pl->skipped->ensure((size_t)std::max(1, pl->npairs) * sizeof(unsigned)));
    P.skipped = pl->skipped->as<unsigned>();
    if (!pl->looked) pl->looked.reset(new DevBuf());
    CK(pl->looked->ensure(sizeof(unsigned long long)));
    P.lookups_skipped = pl->looked->as<unsigned long long>();
    P.trace_on = 0;
    P.bw = bump_words(k);
    pl->smem = cta_smem(t, pl->slice, P.bw);
    int per_sm = 0;
    CK(occupancy(pl->kc, k->score_mode, k->clip_box, pl->block, pl->smem, &per_sm));
    if (per_sm < 1) return fail(ctx, DOCK_ERR_UNSUPPORTED, "tile does not fit on an SM (%zu B shared)", pl->smem);
    int want = (pl->ntask + pl->W - 1) / pl->W;
    pl->grid = std::max(1, std::min(want, per_sm * ctx->num_sms));
    FinalParams& F = pl->F;
    F.pair0 = 0;
    F.lig = P.lig;
    F.pockets = P.pockets;
    F.pose_key = P.pose_key;
    F.pose_xyz = P.pose_xyz;
    F.npairs = pl->npairs;
    F.nlig = B.n;
    F.natoms = B.natoms;
    F.n_poses = N;
    F.shift = k->score_mode == 1 ? 0.0f : 0.5f;
    F.score = ctx->res.as<float>();
    F.xyz_out = ctx->xyz_res.as<float>();
    return DOCK_OK;
}

// Enqueue one batched run: reset the queue, persistent sweep, finalize.
int enqueue_batched(dock_ctx* ctx, Plan* pl, const dock_knobs* k, cudaStream_t s) {
    CK(cudaMemsetAsync(ctx->counter.p, 0, sizeof(unsigned), s));
    if (pl->P.check) CK(cudaMemsetAsync(pl->P.check, 0, sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(pl->skipped->p, 0, (size_t)std::max(1, pl->npairs) * sizeof(unsigned), s));
    CK(cudaMemsetAsync(pl->looked->p, 0, sizeof(unsigned long long), s));
    // external event records become event nodes when this is captured into a graph; outside a
    // capture (the autotuner) they are plain records
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(s, &cs));
    const unsigned flags = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
    CK(cudaEventRecordWithFlags(ctx->ev0, s, flags));
    if (pl->ntask > 0) CK(launch_sweep(pl->kc, pl->P, k->score_mode, k->clip_box, pl->grid, pl->block, pl->smem, s));
    CK(cudaEventRecordWithFlags(ctx->ev1, s, flags));
    if (pl->npairs > 0) {
        finalize_kernel<<<(pl->npairs + 3) / 4, 128, 0, s>>>(pl->F);
        CK(cudaGetLastError());
    }
    return DOCK_OK;
}

// Plain comparison form: per (pocket, ligand) pair, its own queue reset,
// sweep launch over that pair's pose groups, and finalize launch.
int enqueue_plain(dock_ctx* ctx, Plan* pl, const dock_knobs* k, cudaStream_t s) {
    if (pl->P.check) CK(cudaMemsetAsync(pl->P.check, 0, sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(pl->skipped->p, 0, (size_t)std::max(1, pl->npairs) * sizeof(unsigned), s));
    CK(cudaMemsetAsync(pl->looked->p, 0, sizeof(unsigned long long), s));
    CK(cudaEventRecord(ctx->ev0, s));
    for (int pair = 0; pair < pl->npairs; ++pair) {
        SweepParams P = pl->P;
        const int ngroup = pl->task_off[pair + 1] - pl->task_off[pair];
        P.tasks = pl->P.tasks + pl->task_off[pair];
        P.ntask = ngroup;
        int grid = (ngroup + pl->W - 1) / pl->W;
        CK(cudaMemsetAsync(ctx->counter.p, 0, sizeof(unsigned), s));
        CK(launch_sweep(pl->kc, P, k->score_mode, k->clip_box, grid, pl->block, pl->smem, s));
        FinalParams F = pl->F;
        F.pair0 = pair;
        F.npairs = 1;
        finalize_kernel<<<1, 32, 0, s>>>(F);
        CK(cudaGetLastError());
    }
    CK(cudaEventRecord(ctx->ev1, s));
    return DOCK_OK;
}

int check_run_args(dock_ctx* ctx, int batch_id, const int32_t* pids, int np, const dock_knobs* k) {
    if (!ctx) return DOCK_ERR_INVALID_ARG;
    if (batch_id < 0 || batch_id >= (int)ctx->batches.size() || !ctx->batches[batch_id].live)
        return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_run: bad batch id");
    if (np < 1 || !pids) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_run: no pockets");
    for (int i = 0; i < np; ++i)
        if (pids[i] < 0 || pids[i] >= (int)ctx->pockets.size() || !ctx->pockets[pids[i]].live)
            return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_run: bad pocket id %d", pids[i]);
    int rc = check_knobs(ctx, k);
    if (rc) return rc;
    if (k->score_mode == 2)
        for (int i = 0; i < np; ++i)
            if (ctx->pockets[pids[i]].d.npts < 1)
                return fail(ctx, DOCK_ERR_UNSUPPORTED, "exact score: pocket %d was given without probe points", pids[i]);
    int64_t pairs = (int64_t)np * ctx->batches[batch_id].n;
    if (pairs * k->n_poses > (int64_t)1 << 31) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_run: too many poses");
    return DOCK_OK;
}

// Work of one repetition of one pose of ligand b over its 2T sweeps (Alg. 2's
// step choice per sweep): candidates, moving-atom placements, circle bounds
// (every pair once per sweep) and candidate bump pairs.
struct LigWork {
    uint64_t cand = 0, upd = 0, bounds = 0, pairs = 0;
};
LigWork lig_work(const BatchH& B, int b, const dock_knobs* k, const Steps& st) {
    LigWork w;
    for (int s = 0; s < B.nside[b]; ++s) {
        const int si = B.side_off[b] + s;
        const bool coarse = (double)B.side_m[si] / (double)B.l[b] <= k->threshold;
        int phases[2] = {coarse ? st.P_lp - 1 : st.P_hp - 1, 0};
        if (st.tile && !coarse) {
            phases[0] = 360 / st.tile;
            phases[1] = (int)std::lround(st.tile / k->hp_step);
        }
        for (int nc : phases) {
            w.cand += nc;
            w.upd += (uint64_t)nc * B.side_nmov[si];
            w.pairs += (uint64_t)nc * B.side_nmov[si] * B.side_nfixB[si];
        }
        w.bounds += (uint64_t)B.side_nmov[si] * B.side_nfixB[si];
    }
    return w;
}

void count_work(dock_ctx* ctx, const BatchH& B, int np, const dock_knobs* k, const Plan* pl, uint64_t launches) {
    uint64_t cand = 0, upd = 0, bounds = 0, pairs = 0;
    WorkTally& W = ctx->tally;
    W.cand.assign(B.n, 0);
    W.upd.assign(B.n, 0);
    W.bounds.assign(B.n, 0);
    W.pairs.assign(B.n, 0);
    const Steps st = steps_of(k);
    for (int b = 0; b < B.n; ++b) {
        // one repetition of one pose of ligand b
        const LigWork w = lig_work(B, b, k, st);
        W.cand[b] = w.cand;
        W.upd[b] = w.upd;
        W.bounds[b] = w.bounds;
        W.pairs[b] = w.pairs;
        cand += w.cand;
        upd += w.upd;
        bounds += w.bounds;
        pairs += w.pairs;
    }
    W.nlig = B.n;
    W.npairs = np * B.n;
    W.skipped = pl ? pl->skipped.get() : nullptr;
    W.looked = pl ? pl->looked.get() : nullptr;
    W.pending = W.skipped != nullptr;
    uint64_t mult = (uint64_t)np * k->n_poses * k->repetitions;
    ctx->stats.candidates = cand * mult;
    ctx->stats.atom_updates = upd * mult;
    ctx->stats.pair_bounds = bounds * mult;
    ctx->stats.bump_pairs = pairs * mult;
    ctx->stats.kernel_launches = launches;
    ctx->stats.sweep_ms = -1.0;
    ctx->stats.pose_reps_skipped = 0;
    ctx->stats.lookups_skipped = 0;
    ctx->timed = true;
}

}  // namespace

extern "C" {

int dock_run(dock_ctx* ctx, int batch_id, const int32_t* pocket_ids, int npockets, const dock_knobs* k,
             dock_result* out, float* xyz_out, int out_on_device, void* stream) {
    Range range("dock_run");
    int rc = check_run_args(ctx, batch_id, pocket_ids, npockets, k);
    if (rc) return rc;
    if (!out) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_run: NULL out");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    Plan* pl = nullptr;
    if ((rc = get_plan(ctx, batch_id, pocket_ids, npockets, k, k->plain_mode, &pl))) return rc;
    const BatchH& B = ctx->batches[batch_id];
    uint64_t launches = 0;
    if (k->plain_mode) {
        if ((rc = enqueue_plain(ctx, pl, k, s))) return rc;
        launches = 2ull * pl->npairs;
    } else {
        if (!pl->exec || pl->exec_stream != s) {
            // capture the batched run once per plan and replay it
            if (pl->exec) {
                cudaGraphExecDestroy(pl->exec);
                pl->exec = nullptr;
            }
            cudaStream_t cap = s;
            cudaStream_t own = nullptr;
            if (!cap) {
                CK(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
                cap = own;
            }
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
            int erc = enqueue_batched(ctx, pl, k, cap);
            cudaError_t ce = cudaStreamEndCapture(cap, &g);
            if (own) cudaStreamDestroy(own);
            if (erc) {
                if (g) cudaGraphDestroy(g);
                return erc;
            }
            CK(ce);
            cudaError_t ie = cudaGraphInstantiate(&pl->exec, g, 0);
            cudaGraphDestroy(g);
            CK(ie);
            pl->exec_stream = s;
        }
        CK(cudaGraphLaunch(pl->exec, s));
        launches = (pl->ntask > 0 ? 1 : 0) + (pl->npairs > 0 ? 1 : 0);
    }
    const size_t rbytes = (size_t)pl->npairs * sizeof(dock_result);
    const size_t xbytes = (size_t)npockets * B.natoms * 3 * sizeof(float);
    cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (rbytes) CK(cudaMemcpyAsync(out, ctx->res.p, rbytes, kind, s));
    if (xyz_out && xbytes) CK(cudaMemcpyAsync(xyz_out, ctx->xyz_res.p, xbytes, kind, s));
    if (!out_on_device) CK(cudaStreamSynchronize(s));
    count_work(ctx, B, npockets, k, pl, launches);
    return read_check(ctx, s);
}

}  // extern "C"

namespace {

// Wait for a pipeline stage's chunk, scatter its results into the caller's
// arrays (pair = pocket * n + ligand; coordinates pocket-major) and add its
// work, less the repetitions left out at fixed points, to the totals.
int finish_chunk(dock_ctx* ctx, DbSlot& S, const dock_ligand_batch* b, int np, const dock_knobs* k,
                 dock_result* out, float* xyz_out, dock_stats& tot) {
    CK(cudaEventSynchronize(S.done));
    S.pending = false;
    const int n = b->n, nc = S.c1 - S.c0;
    const int natoms = b->atom_off[n];
    const int a0 = b->atom_off[S.c0], na = b->atom_off[S.c1] - a0;
    const dock_result* r = static_cast<const dock_result*>(S.hres);
    for (int pk = 0; pk < np; ++pk) std::memcpy(out + (size_t)pk * n + S.c0, r + (size_t)pk * nc, nc * sizeof(dock_result));
    if (xyz_out)
        for (int pk = 0; pk < np; ++pk)
            std::memcpy(xyz_out + ((size_t)pk * natoms + a0) * 3, static_cast<const float*>(S.hxyz) + (size_t)pk * na * 3,
                        (size_t)na * 3 * sizeof(float));
    const unsigned* sk = static_cast<const unsigned*>(S.hskip);
    const unsigned long long gated = *static_cast<const unsigned long long*>(S.hlook);
    tot.lookups_skipped += gated;
    tot.atom_updates -= gated;
    const uint64_t mult = (uint64_t)k->n_poses * k->repetitions;
    const Steps st = steps_of(k);
    for (int i = 0; i < nc; ++i) {
        const LigWork w = lig_work(S.B, i, k, st);
        for (int pk = 0; pk < np; ++pk) {
            const uint64_t reps = mult - sk[(size_t)pk * nc + i];
            tot.candidates += reps * w.cand;
            tot.atom_updates += reps * w.upd;
            tot.pair_bounds += reps * w.bounds;
            tot.bump_pairs += reps * w.pairs;
            tot.pose_reps_skipped += sk[(size_t)pk * nc + i];
        }
    }
    return DOCK_OK;
}

}  // namespace

extern "C" {

int dock_measure_peaks(dock_ctx* ctx, int pocket_id, dock_peaks* out, void* stream) {
    if (!ctx) return DOCK_ERR_INVALID_ARG;
    if (!out) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_measure_peaks: NULL out");
    if (pocket_id < 0 || pocket_id >= (int)ctx->pockets.size() || !ctx->pockets[pocket_id].live)
        return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_measure_peaks: bad pocket id %d", pocket_id);
    CK(cudaSetDevice(ctx->device));
    const PocketH& ph = ctx->pockets[pocket_id];
    double r[5] = {0, 0, 0, 0, 0};
    CK(gd::measure_peaks(ph.Kt->tex, ph.d.nx + 2 * PAD, ph.d.ny + 2 * PAD, ph.d.nz + 2 * PAD, ctx->num_sms,
                         (cudaStream_t)stream, r));
    out->fma_per_s = r[0];
    out->ffma2_per_s = r[1];
    out->tex_field_per_s = r[2];
    out->tex_local_per_s = r[3];
    out->l2_sectors_per_s = r[4];
    return DOCK_OK;
}

int dock_run_database(dock_ctx* ctx, const dock_ligand_batch* b, const int32_t* pocket_ids, int npockets,
                      const dock_knobs* k, int chunk, dock_result* out, float* xyz_out, void* stream) {
    Range range("dock_run_database");
    if (!ctx) return DOCK_ERR_INVALID_ARG;
    if (!b || !out) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_run_database: NULL argument");
    if (chunk < 1) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_run_database: chunk < 1");
    if (npockets < 1 || !pocket_ids) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_run_database: no pockets");
    for (int i = 0; i < npockets; ++i)
        if (pocket_ids[i] < 0 || pocket_ids[i] >= (int)ctx->pockets.size() || !ctx->pockets[pocket_ids[i]].live)
            return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_run_database: bad pocket id %d", pocket_ids[i]);
    int rc = check_knobs(ctx, k);
    if (rc) return rc;
    if (k->score_mode == 2)
        for (int i = 0; i < npockets; ++i)
            if (ctx->pockets[pocket_ids[i]].d.npts < 1)
                return fail(ctx, DOCK_ERR_UNSUPPORTED, "exact score: pocket %d was given without probe points",
                            pocket_ids[i]);
    if (b->n < 0) return fail(ctx, DOCK_ERR_INVALID_ARG, "batch: n < 0");
    const int n = b->n;
    ctx->stats = dock_stats{};
    ctx->tally.pending = false;
    ctx->timed = false;
    ctx->stats.sweep_ms = -1.0;
    if (n == 0) return DOCK_OK;
    if (!b->atom_off || !b->xyz || !b->bond_off || !b->rot_off)
        return fail(ctx, DOCK_ERR_INVALID_ARG, "batch: NULL array");
    if (b->atom_off[0] != 0 || b->bond_off[0] != 0 || b->rot_off[0] != 0)
        return fail(ctx, DOCK_ERR_INVALID_ARG, "batch: offsets must start at 0");
    for (int i = 0; i < n; ++i)
        if (b->atom_off[i + 1] < b->atom_off[i] || b->bond_off[i + 1] < b->bond_off[i] || b->rot_off[i + 1] < b->rot_off[i])
            return fail(ctx, DOCK_ERR_INVALID_ARG, "batch: offsets must not decrease (ligand %d)", i);
    chunk = std::min(chunk, n);
    if ((int64_t)npockets * chunk * k->n_poses > (int64_t)1 << 31)
        return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_run_database: too many poses per chunk");
    CK(cudaSetDevice(ctx->device));
    const int nchunk = (n + chunk - 1) / chunk;
    int max_atoms = 0;
    for (int c = 0; c < nchunk; ++c)
        max_atoms = std::max(max_atoms, b->atom_off[std::min(n, (c + 1) * chunk)] - b->atom_off[c * chunk]);
    if ((rc = ensure_scratch(ctx, npockets, chunk, max_atoms, k->n_poses))) return rc;
    if (!ctx->copy) CK(cudaStreamCreateWithFlags(&ctx->copy, cudaStreamNonBlocking));
    for (DbSlot& S : ctx->db) {
        // a call that failed part way may have left copies in flight into these buffers
        if (S.pending) CK(cudaEventSynchronize(S.done));
        S.pending = false;
        if (!S.up) CK(cudaEventCreateWithFlags(&S.up, cudaEventDisableTiming));
        if (!S.done) CK(cudaEventCreateWithFlags(&S.done, cudaEventDisableTiming));
    }
    const cudaStream_t s = (cudaStream_t)stream;
    dock_tile t = default_tile(k);
    if (ctx->tile.lanes_per_pose) t.lanes_per_pose = ctx->tile.lanes_per_pose;
    if (ctx->tile.angles_per_chunk) t.angles_per_chunk = ctx->tile.angles_per_chunk;
    if (ctx->tile.warps_per_cta) t.warps_per_cta = ctx->tile.warps_per_cta;
    if (k->score_mode == 2) t.angles_per_chunk = 12;
    dock_stats tot{};
    uint64_t launches = 0;
    // Chunk i is prepared on the host while the device sweeps chunk i-1; its
    // upload runs on the copy stream, its sweep, finalize and result copies on
    // the caller's stream; the results of chunk i-1 are collected after chunk i
    // is enqueued, so the device always has the next chunk waiting.
    for (int c = 0; c < nchunk; ++c) {
        DbSlot& S = ctx->db[c & 1];
        if (S.pending && (rc = finish_chunk(ctx, S, b, npockets, k, out, xyz_out, tot))) return rc;
        S.c0 = c * chunk;
        S.c1 = std::min(n, S.c0 + chunk);
        const int nc = S.c1 - S.c0;
        const int a0 = b->atom_off[S.c0], e0 = b->bond_off[S.c0], r0 = b->rot_off[S.c0];
        S.aoff.resize(nc + 1);
        S.boff.resize(nc + 1);
        S.roff.resize(nc + 1);
        for (int i = 0; i <= nc; ++i) {
            S.aoff[i] = b->atom_off[S.c0 + i] - a0;
            S.boff[i] = b->bond_off[S.c0 + i] - e0;
            S.roff[i] = b->rot_off[S.c0 + i] - r0;
        }
        dock_ligand_batch v = *b;
        v.n = nc;
        v.atom_off = S.aoff.data();
        v.xyz = b->xyz + (size_t)3 * a0;
        v.bond_off = S.boff.data();
        v.bonds = b->bonds ? b->bonds + (size_t)2 * e0 : nullptr;
        v.rot_off = S.roff.data();
        v.rot = b->rot ? b->rot + r0 : nullptr;
        v.id_base = b->id_base + S.c0;
        v.ids = b->ids ? b->ids + S.c0 : nullptr;
        nvtxRangePushA("database chunk: host preparation");
        rc = prep_batch(ctx, &v, S.B, S.im);
        nvtxRangePop();
        if (rc) {
            // a bad ligand in chunk c: report it by its index in the database
            ctx->err = "ligands " + std::to_string(S.c0) + ".." + std::to_string(S.c1 - 1) + ": " + ctx->err;
            for (DbSlot& o : ctx->db)
                if (o.pending) cudaEventSynchronize(o.done), o.pending = false;
            return rc;
        }
        // headroom so that later chunks rarely grow the buffers (growing synchronizes)
        const size_t total = S.im.total + S.im.total / 4;
        if ((rc = ensure_pinned(ctx, &S.stage, &S.stage_bytes, total))) return rc;
        stage_batch(S.im, S.B.natoms, static_cast<uint8_t*>(S.stage));
        if (!S.mem) S.mem.reset(new DevBuf());
        if (S.mem->n < S.im.total) CK(S.mem->ensure(total));
        CK(cudaMemcpyAsync(S.mem->p, S.stage, S.im.total, cudaMemcpyHostToDevice, ctx->copy));
        bind_batch(S.B, S.im, S.mem->as<uint8_t>());
        S.B.live = true;
        if ((rc = build_plan(ctx, S.B, pocket_ids, npockets, k, t, 0, &S.plan, ctx->copy))) return rc;
        CK(cudaEventRecord(S.up, ctx->copy));
        CK(cudaStreamWaitEvent(s, S.up, 0));
        if ((rc = enqueue_batched(ctx, &S.plan, k, s))) return rc;
        launches += (S.plan.ntask > 0 ? 1 : 0) + (S.plan.npairs > 0 ? 1 : 0);
        const size_t rbytes = (size_t)npockets * nc * sizeof(dock_result);
        const size_t xbytes = (size_t)npockets * S.B.natoms * 3 * sizeof(float);
        const size_t kbytes = (size_t)npockets * nc * sizeof(unsigned);
        if ((rc = ensure_pinned(ctx, &S.hres, &S.hres_bytes, rbytes + rbytes / 4))) return rc;
        if ((rc = ensure_pinned(ctx, &S.hskip, &S.hskip_bytes, kbytes + kbytes / 4))) return rc;
        CK(cudaMemcpyAsync(S.hres, ctx->res.p, rbytes, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(S.hskip, S.plan.skipped->p, kbytes, cudaMemcpyDeviceToHost, s));
        if ((rc = ensure_pinned(ctx, &S.hlook, &S.hlook_bytes, sizeof(unsigned long long)))) return rc;
        CK(cudaMemcpyAsync(S.hlook, S.plan.looked->p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        if (xyz_out && xbytes) {
            if ((rc = ensure_pinned(ctx, &S.hxyz, &S.hxyz_bytes, xbytes + xbytes / 4))) return rc;
            CK(cudaMemcpyAsync(S.hxyz, ctx->xyz_res.p, xbytes, cudaMemcpyDeviceToHost, s));
        }
        CK(cudaEventRecord(S.done, s));
        S.pending = true;
        DbSlot& prev = ctx->db[(c + 1) & 1];
        if (prev.pending && (rc = finish_chunk(ctx, prev, b, npockets, k, out, xyz_out, tot))) return rc;
    }
    for (DbSlot& S : ctx->db)
        if (S.pending && (rc = finish_chunk(ctx, S, b, npockets, k, out, xyz_out, tot))) return rc;
    tot.kernel_launches = launches;
    tot.sweep_ms = -1.0;
    ctx->stats = tot;
    return read_check(ctx, s);
}

int dock_run_trace(dock_ctx* ctx, int batch_id, int pocket_id, const dock_knobs* k, const dock_trace* tr,
                   dock_result* out, void* stream) {
    Range range("dock_run_trace");
    int rc = check_run_args(ctx, batch_id, &pocket_id, 1, k);
    if (rc) return rc;
    if (!tr || !tr->chosen_k || !tr->cand_S || !tr->cand_status || !tr->pose_S || !tr->pose_init_S ||
        !tr->pose_status || !tr->init_xyz || !tr->pose_xyz)
        return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_run_trace: NULL trace buffer");
    if (tr->pmax < trace_pmax(k)) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_run_trace: pmax too small");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    Plan* pl = nullptr;
    int32_t pid = pocket_id;
    if ((rc = get_plan(ctx, batch_id, &pid, 1, k, 0, &pl))) return rc;
    SweepParams P = pl->P;
    P.trace_on = 1;
    P.skipped = nullptr;  // the plan's work counters belong to dock_run
    P.lookups_skipped = nullptr;
    P.tr.pmax = tr->pmax;
    P.tr.chosen_k = tr->chosen_k;
    P.tr.cand_S = tr->cand_S;
    P.tr.cand_status = tr->cand_status;
    P.tr.pose_S = tr->pose_S;
    P.tr.pose_init_S = tr->pose_init_S;
    P.tr.pose_status = tr->pose_status;
    P.tr.init_xyz = tr->init_xyz;
    P.tr.pose_xyz = tr->pose_xyz;
    CK(cudaMemsetAsync(ctx->counter.p, 0, sizeof(unsigned), s));
    if (P.check) CK(cudaMemsetAsync(P.check, 0, sizeof(unsigned long long), s));
    if (pl->ntask > 0) CK(launch_sweep(pl->kc, P, k->score_mode, k->clip_box, pl->grid, pl->block, pl->smem, s));
    if (pl->npairs > 0) {
        finalize_kernel<<<(pl->npairs + 3) / 4, 128, 0, s>>>(pl->F);
        CK(cudaGetLastError());
    }
    if (out && pl->npairs)
        CK(cudaMemcpyAsync(out, ctx->res.p, (size_t)pl->npairs * sizeof(dock_result), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return read_check(ctx, s);
}

int dock_autotune(dock_ctx* ctx, int batch_id, int pocket_id, const dock_knobs* k, dock_tile* best, void* stream) {
    Range range("dock_autotune");
    int32_t pid = pocket_id;
    int rc = check_run_args(ctx, batch_id, &pid, 1, k);
    if (rc) return rc;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const dock_tile saved = ctx->tile;
    const std::string tkey = plan_key(batch_id, nullptr, 0, k, dock_tile{0, 0, 0}, 0);
    ctx->tuned.erase(tkey);
    std::vector<int> Qs;
    for (int q : {1, 2, 4, 8})
        if (32 / q <= 2 * k->n_poses || q == 8) Qs.push_back(q);
    std::vector<int> kcs{8, 12, 18, 36};
    if (k->score_mode == 2) kcs = {12};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    dock_tile bt = default_tile(k);
    for (int q : Qs)
        for (int kc : kcs)
            for (int w : {2, 4, 8}) {
                dock_tile t{q, kc, w};
                ctx->tile = t;
                Plan* pl = nullptr;
                if (get_plan(ctx, batch_id, &pid, 1, k, 0, &pl)) continue;
                float ms = 0;
                bool ok = true;
                for (int rep = 0; rep < 2 && ok; ++rep) {  // first pass warms up
                    cudaEventRecord(e0, s);
                    ok = enqueue_batched(ctx, pl, k, s) == DOCK_OK;
                    cudaEventRecord(e1, s);
                    ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
                    ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
                }
                if (!ok) {
                    // a shape this device cannot run: drop its error and its plan, keep going
                    cudaStreamSynchronize(s);
                    cudaGetLastError();
                }
                if (ok && ms < best_ms) {
                    best_ms = ms;
                    bt = t;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tile = saved;
    ctx->err.clear();
    ctx->tuned[tkey] = bt;
    if (best) *best = bt;
    return DOCK_OK;
}

}  // extern "C"

// ======================================================== static-scratch run
//
// dock_run_static: the batched sweep with its scratch (work-queue head, angle
// tables, task list, per-pose keys and coordinates) taken from one file-scope
// device array instead of allocated memory. The array is created when the
// library's module is loaded on a device and held there until the process
// exits, whether or not this entry point is ever called. Nothing of the call
// goes through host memory after it is enqueued: the angle tables travel as
// kernel parameters, the pocket descriptor is the one dock_init_pocket left
// on the device, and the step choice of Alg. 2 is made in the sweep kernel.

namespace {

constexpr int64_t kStaticPoseSlots = int64_t(1) << 17;  // (ligand, pose) slots per call
constexpr int64_t kStaticAtomPoses = int64_t(1) << 22;  // (atom, pose) slots per call
constexpr int kStaticAngles = 361;                       // angles per table (1 degree steps and up)

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffCounter = 0;
constexpr size_t kOffCheck = 8;  // status word of the index checks (checked builds)
constexpr size_t kOffTables = 256;
constexpr size_t kOffTasks = kOffTables + align256(3 * kStaticAngles * sizeof(float2));
constexpr size_t kOffKeys = kOffTasks + align256(kStaticPoseSlots * sizeof(int2));
constexpr size_t kOffXyz = kOffKeys + align256(kStaticPoseSlots * sizeof(unsigned long long));
constexpr size_t kStaticBytes = kOffXyz + align256(kStaticAtomPoses * 3 * sizeof(float));  // about 50 MiB

}  // namespace

static __device__ __align__(256) unsigned char g_dock_scratch[kStaticBytes];

namespace {

// Device address of g_dock_scratch on each device, looked up once per device
// (with that device current) on the first call there. It stays valid for the
// life of the device's primary context.
std::mutex g_static_mu;
void* g_static_addr[256] = {};

cudaError_t static_scratch(int device, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (device < 0 || device >= 256) return cudaErrorInvalidDevice;
    if (!g_static_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_dock_scratch);
        if (e != cudaSuccess) return e;
        g_static_addr[device] = p;
    }
    *out = static_cast<unsigned char*>(g_static_addr[device]);
    return cudaSuccess;
}

// The run's angle tables (cos, sin) by value: hp, lp and tile centres.
struct StaticTables {
    float2 t[3][kStaticAngles];
};

// Set-up of one call, in stream order before the sweep: the queue head to
// zero, the angle tables into the array, and the work list in (pocket-ligand
// pair, pose group) order with each ligand's lanes per pose chosen as the
// batched form chooses them (the smallest power of two >= lq0 whose pose
// group of 32 >> lq poses fits the warp's coordinate slice). Every ligand
// gets ngroup slots; a group past its ligand's poses is an idle task.
__global__ void static_setup_kernel(const __grid_constant__ StaticTables tabs, unsigned* counter,
                                    unsigned long long* check, float2* tab_out, int2* tasks, const LigDev* lig,
                                    int nlig, int ngroup, int lq0, int slice) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        *counter = 0u;
        *check = 0ull;
    }
    if (t < 3 * kStaticAngles) tab_out[t] = tabs.t[t / kStaticAngles][t % kStaticAngles];
    if (t < (int64_t)nlig * ngroup) {
        const int b = (int)(t / ngroup), g = (int)(t % ngroup);
        const int l = lig[b].l;
        int lq = lq0;
        while (lq < 5 && (32 >> lq) * l * 3 > slice) ++lq;
        tasks[t] = make_int2(b, g | (lq << 16));
    }
}

// cos/sin of the angles offset + i * stride (degrees), FP64 rounded to FP32
// (the same values as the batched form's tables).
void fill_table(float2* t, int n, double offset, double stride) {
    const double rad = 3.14159265358979323846 / 180.0;
    for (int i = 0; i < n; ++i) {
        double a = offset + i * stride;
        t[i] = make_float2((float)std::cos(a * rad), (float)std::sin(a * rad));
    }
}

}  // namespace

extern "C" int dock_run_static(dock_ctx* ctx, int batch_id, int pocket_id, const dock_knobs* k, dock_result* out,
                               float* xyz_out, void* stream) {
    int32_t pid = pocket_id;
    int rc = check_run_args(ctx, batch_id, &pid, 1, k);
    if (rc) return rc;
    if (!out) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_run_static: NULL out");
    CK(cudaSetDevice(ctx->device));
    const BatchH& B = ctx->batches[batch_id];
    const int N = k->n_poses;
    const int64_t pose_slots = (int64_t)B.n * N, atom_poses = (int64_t)B.natoms * N;
    if (pose_slots > kStaticPoseSlots || atom_poses > kStaticAtomPoses)
        return fail(ctx, DOCK_ERR_INVALID_ARG,
                    "dock_run_static: %lld ligand-poses and %lld atom-poses exceed the static scratch "
                    "(at most %lld and %lld per call); split the batch or use dock_run",
                    (long long)pose_slots, (long long)atom_poses, (long long)kStaticPoseSlots,
                    (long long)kStaticAtomPoses);
    const int P_hp = n_angles(k->hp_step), P_lp = n_angles(k->lp_step);
    int n_tiles = 0, per_tile = 0, tile = 0;
    if (k->enable_refinement) {
        tile = peel_tile(k->hp_step);
        n_tiles = 360 / tile;
        per_tile = (int)std::lround(tile / k->hp_step);
    }
    if (P_hp > kStaticAngles || P_lp > kStaticAngles || n_tiles > kStaticAngles)
        return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_run_static: too many angles per sweep");
    unsigned char* base = nullptr;
    CK(static_scratch(ctx->device, &base));
    cudaStream_t s = (cudaStream_t)stream;

    // tile shape: the forced fields of dock_set_tile over the default (an autotuned shape is not used)
    dock_tile t = default_tile(k);
    if (ctx->tile.lanes_per_pose) t.lanes_per_pose = ctx->tile.lanes_per_pose;
    if (ctx->tile.angles_per_chunk) t.angles_per_chunk = ctx->tile.angles_per_chunk;
    if (ctx->tile.warps_per_cta) t.warps_per_cta = ctx->tile.warps_per_cta;
    if (k->score_mode == 2) t.angles_per_chunk = 12;
    const int slice = slice_floats(t, B.lmax);
    int lq0 = 0;
    while ((1 << lq0) < t.lanes_per_pose) ++lq0;
    const int lq_max = lanes_log2(t, slice, B.lmax);  // the largest ligand has the fewest poses per warp
    const int W = t.warps_per_cta, block = 32 * W;
    const int ngroup = (N + (32 >> lq_max) - 1) / (32 >> lq_max);
    const int ntask = B.n * ngroup;
    const int bw = bump_words(k);
    const size_t smem = cta_smem(t, slice, bw);
    int per_sm = 0;
    CK(occupancy(t.angles_per_chunk, k->score_mode, k->clip_box, block, smem, &per_sm));
    if (per_sm < 1) return fail(ctx, DOCK_ERR_UNSUPPORTED, "dock_run_static: tile does not fit on an SM");

    // set-up in stream order: queue head, angle tables (kernel parameters), work list
    StaticTables tabs;
    fill_table(tabs.t[0], P_hp, 0.0, k->hp_step);
    fill_table(tabs.t[1], P_lp, 0.0, k->lp_step);
    if (n_tiles) fill_table(tabs.t[2], n_tiles, 0.5 * tile, (double)tile);
    else tabs.t[2][0] = make_float2(1.f, 0.f);
    float2* tab = reinterpret_cast<float2*>(base + kOffTables);
    const int64_t nset = std::max<int64_t>(3 * kStaticAngles, ntask);
    static_setup_kernel<<<(unsigned)((nset + 255) / 256), 256, 0, s>>>(
        tabs, reinterpret_cast<unsigned*>(base + kOffCounter), reinterpret_cast<unsigned long long*>(base + kOffCheck),
        tab, reinterpret_cast<int2*>(base + kOffTasks), B.d_lig, B.n, ngroup, lq0, slice);
    CK(cudaGetLastError());

    const PocketDev* pdev = ctx->pockets[pocket_id].dev->as<PocketDev>();
    SweepParams P{};
    P.lig = B.d_lig;
    P.side = B.d_side;
    P.idx = B.d_idx;
    P.xyz0 = B.d_xyz0;
    P.pockets = pdev;
    P.tasks = reinterpret_cast<const int2*>(base + kOffTasks);
    P.ntask = ntask;
    P.npockets = 1;
    P.nidx = B.nidx;
#ifdef GEODOCK_CHECKED
    P.check = reinterpret_cast<unsigned long long*>(base + kOffCheck);
#endif
    P.nlig = B.n;
    P.natoms = B.natoms;
    P.counter = reinterpret_cast<unsigned*>(base + kOffCounter);
    P.n_poses = N;
    P.repetitions = k->repetitions;
    P.slice = slice;
    P.bw = bw;
    P.threshold = k->threshold;
    P.coarse = nullptr;  // Alg. 2's step choice per sweep in the kernel (the same FP64 test as on the host)
    P.bump_thr = k->bump_thr;
    P.seed = k->seed;
    P.cs_hp = tab;
    P.cs_lp = tab + kStaticAngles;
    P.P_hp = P_hp;
    P.P_lp = P_lp;
    P.peel = k->enable_refinement ? 1 : 0;
    P.hp_step = (float)k->hp_step;
    P.lp_step = (float)k->lp_step;
    P.tile = (float)tile;
    P.cs_peel = tab + 2 * kStaticAngles;
    P.n_tiles = n_tiles;
    P.per_tile = per_tile;
    P.pose_key = reinterpret_cast<unsigned long long*>(base + kOffKeys);
    P.pose_xyz = reinterpret_cast<float*>(base + kOffXyz);
    P.trace_on = 0;
    if (ntask > 0) {
        const int grid = std::max(1, std::min((ntask + W - 1) / W, per_sm * ctx->num_sms));
        CK(launch_sweep(t.angles_per_chunk, P, k->score_mode, k->clip_box, grid, block, smem, s));
    }
    if (B.n > 0) {
        FinalParams F{};
        F.pair0 = 0;
        F.lig = P.lig;
        F.pockets = pdev;
        F.pose_key = P.pose_key;
        F.pose_xyz = P.pose_xyz;
        F.npairs = B.n;
        F.nlig = B.n;
        F.natoms = B.natoms;
        F.n_poses = N;
        F.shift = k->score_mode == 1 ? 0.0f : 0.5f;
        F.score = reinterpret_cast<float*>(out);
        F.xyz_out = xyz_out;
        finalize_kernel<<<(B.n + 3) / 4, 128, 0, s>>>(F);
        CK(cudaGetLastError());
    }
    // checked builds wait here and report a failed index check
    return read_check(ctx, s, P.check);
}

// ------------------------------------------------------------ local refinement

namespace {

int check_batch(dock_ctx* ctx, int batch_id) {
    if (!ctx) return DOCK_ERR_INVALID_ARG;
    if (batch_id < 0 || batch_id >= (int)ctx->batches.size() || !ctx->batches[batch_id].live)
        return fail(ctx, DOCK_ERR_INVALID_ARG, "bad batch id");
    return DOCK_OK;
}

int check_pocket(dock_ctx* ctx, int pocket_id) {
    if (pocket_id < 0 || pocket_id >= (int)ctx->pockets.size() || !ctx->pockets[pocket_id].live)
        return fail(ctx, DOCK_ERR_INVALID_ARG, "bad pocket id %d", pocket_id);
    return DOCK_OK;
}

BatchBounds bounds_of(dock_ctx* ctx, const BatchH& B) {
    BatchBounds bb{};
    bb.natoms = B.natoms;
    bb.nside = B.nside_total;
    bb.nidx = B.nidx;
    bb.ntor = B.ntor;
    bb.nchk = B.nchk;
    bb.lmax = B.lmax;
    bb.check = check_word(ctx);
    return bb;
}

ScoreParams score_params(dock_ctx* ctx, const BatchH& B, const PocketDev* pocket_dev) {
    ScoreParams P{};
    P.bounds = bounds_of(ctx, B);
    P.lig = B.d_lig;
    P.side = B.d_side;
    P.idx = B.d_idx;
    P.rlig = B.d_rlig;
    P.rtor = B.d_rtor;
    P.pocket = pocket_dev;
    P.nlig = B.n;
    return P;
}

// Device descriptor of one pocket (written once at dock_init_pocket).
int pocket_on_device(dock_ctx* ctx, int pocket_id, cudaStream_t s, const PocketDev** out) {
    (void)s;
    *out = ctx->pockets[pocket_id].dev->as<PocketDev>();
    return DOCK_OK;
}

// Device array of the descriptors of a pocket list, built once per list.
int pocket_set(dock_ctx* ctx, const int32_t* pids, int np, const PocketDev** out) {
    std::string key;
    for (int i = 0; i < np; ++i) key += std::to_string(pids[i]) + ",";
    auto it = ctx->pocket_sets.find(key);
    if (it == ctx->pocket_sets.end()) {
        std::vector<PocketDev> pd(np);
        for (int i = 0; i < np; ++i) pd[i] = ctx->pockets[pids[i]].d;
        std::unique_ptr<DevBuf> buf(new DevBuf());
        CK(buf->ensure(np * sizeof(PocketDev)));
        CK(cudaMemcpy(buf->p, pd.data(), np * sizeof(PocketDev), cudaMemcpyHostToDevice));
        it = ctx->pocket_sets.emplace(key, std::move(buf)).first;
    }
    *out = it->second->as<PocketDev>();
    return DOCK_OK;
}

int refine_impl(dock_ctx* ctx, int batch_id, const int32_t* pids, int np, const dock_knobs* k, const float* xyz_in,
                dock_result* out, float* xyz_out, int on_device, const dock_refine_trace_buf* tr, cudaStream_t s) {
    Range range("dock_refine");
    int rc = check_run_args(ctx, batch_id, pids, np, k);
    if (rc) return rc;
    if (!xyz_in || !out || !xyz_out) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_refine: NULL buffer");
    CK(cudaSetDevice(ctx->device));
    const BatchH& B = ctx->batches[batch_id];
    const int npairs = np * B.n;
    const size_t xbytes = (size_t)np * B.natoms * 3 * sizeof(float);
    const PocketDev* pset = nullptr;
    if ((rc = pocket_set(ctx, pids, np, &pset))) return rc;
    const float* xin = xyz_in;
    float* xout = xyz_out;
    float* res = reinterpret_cast<float*>(out);
    if (!on_device) {
        CK(ctx->ref_xyz_in.ensure(std::max<size_t>(xbytes, 16)));
        CK(ctx->ref_xyz_out.ensure(std::max<size_t>(xbytes, 16)));
        CK(ctx->ref_res.ensure(std::max<size_t>((size_t)npairs * sizeof(dock_result), 16)));
        if (xbytes) CK(cudaMemcpyAsync(ctx->ref_xyz_in.p, xyz_in, xbytes, cudaMemcpyHostToDevice, s));
        xin = ctx->ref_xyz_in.as<float>();
        xout = ctx->ref_xyz_out.as<float>();
        res = ctx->ref_res.as<float>();
    }
    RefineParams P{};
    P.lig = B.d_lig;
    P.side = B.d_side;
    P.idx = B.d_idx;
    P.rlig = B.d_rlig;
    P.rtor = B.d_rtor;
    P.check = B.d_check;
    P.pockets = pset;
    P.npairs = npairs;
    P.nlig = B.n;
    P.natoms = B.natoms;
    P.steps = k->refine_steps;
    P.clip = k->clip_box;
    P.thr2 = (float)(k->bump_thr * k->bump_thr);
    P.xyz_in = xin;
    P.xyz_out = xout;
    P.result = res;
    P.bounds = bounds_of(ctx, B);
    std::vector<DevBuf> tbuf(10);
    const int ns = npairs * k->refine_steps;
    if (tr) {
        if (tr->gstride < 6 + B.tmax) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_refine_trace: gstride too small");
        P.trace_on = 1;
        P.tr.gstride = tr->gstride;
        size_t sz[10] = {(size_t)ns * tr->gstride * 4, (size_t)ns * 4, (size_t)ns * 4, (size_t)ns * 4, (size_t)ns * 4,
                         (size_t)ns * 4, (size_t)npairs * 4, (size_t)npairs * 4, (size_t)npairs * 4, 0};
        for (int i = 0; i < 9; ++i) {
            CK(tbuf[i].ensure(std::max<size_t>(sz[i], 16)));
            CK(cudaMemsetAsync(tbuf[i].p, 0, std::max<size_t>(sz[i], 16), s));
        }
        P.tr.G = tbuf[0].as<float>();
        P.tr.D = tbuf[1].as<float>();
        P.tr.lam = tbuf[2].as<float>();
        P.tr.S_new = tbuf[3].as<float>();
        P.tr.verdict = tbuf[4].as<int32_t>();
        P.tr.accept = tbuf[5].as<int32_t>();
        P.tr.S_start = tbuf[6].as<float>();
        P.tr.S_final = tbuf[7].as<float>();
        P.tr.status = tbuf[8].as<int32_t>();
    }
    CK(launch_refine(P, B.lmax, B.tmax, s));
    if ((rc = read_check(ctx, s))) return rc;
    if (tr) {
        CK(cudaStreamSynchronize(s));
        CK(cudaMemcpy(tr->G, P.tr.G, (size_t)ns * tr->gstride * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(tr->D, P.tr.D, (size_t)ns * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(tr->lam, P.tr.lam, (size_t)ns * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(tr->S_new, P.tr.S_new, (size_t)ns * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(tr->verdict, P.tr.verdict, (size_t)ns * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(tr->accept, P.tr.accept, (size_t)ns * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(tr->S_start, P.tr.S_start, (size_t)npairs * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(tr->S_final, P.tr.S_final, (size_t)npairs * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(tr->status, P.tr.status, (size_t)npairs * 4, cudaMemcpyDeviceToHost));
    }
    if (!on_device) {
        if (npairs) CK(cudaMemcpyAsync(out, res, (size_t)npairs * sizeof(dock_result), cudaMemcpyDeviceToHost, s));
        if (xbytes) CK(cudaMemcpyAsync(xyz_out, xout, xbytes, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return DOCK_OK;
}

}  // namespace

extern "C" {

int dock_batch_info(dock_ctx* ctx, int batch_id, int* n, int* natoms, int* lmax, int* tmax) {
    int rc = check_batch(ctx, batch_id);
    if (rc) return rc;
    const BatchH& B = ctx->batches[batch_id];
    if (n) *n = B.n;
    if (natoms) *natoms = B.natoms;
    if (lmax) *lmax = B.lmax;
    if (tmax) *tmax = B.tmax;
    return DOCK_OK;
}

int dock_score_trilinear(dock_ctx* ctx, int batch_id, int pocket_id, int clip, const float* xyz, float* o,
                         void* stream) {
    int rc = check_batch(ctx, batch_id);
    if (rc || (rc = check_pocket(ctx, pocket_id))) return rc;
    if (!xyz || !o) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_score_trilinear: NULL buffer");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const PocketDev* pdev = nullptr;
    if ((rc = pocket_on_device(ctx, pocket_id, s, &pdev))) return rc;
    const BatchH& B = ctx->batches[batch_id];
    ScoreParams P = score_params(ctx, B, pdev);
    P.clip = clip != 0;
    P.x = xyz;
    P.out = o;
    CK(launch_score(P, B.lmax, SCORE_FWD, s));
    return read_check(ctx, s);
}

int dock_score_trilinear_grad(dock_ctx* ctx, int batch_id, int pocket_id, int clip, const float* xyz,
                              const float* grad_o, float* grad_xyz, void* stream) {
    int rc = check_batch(ctx, batch_id);
    if (rc || (rc = check_pocket(ctx, pocket_id))) return rc;
    if (!xyz || !grad_xyz) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_score_trilinear_grad: NULL buffer");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const PocketDev* pdev = nullptr;
    if ((rc = pocket_on_device(ctx, pocket_id, s, &pdev))) return rc;
    const BatchH& B = ctx->batches[batch_id];
    ScoreParams P = score_params(ctx, B, pdev);
    P.clip = clip != 0;
    P.x = xyz;
    P.grad_in = grad_o;
    P.out = grad_xyz;
    CK(launch_score(P, B.lmax, SCORE_BWD, s));
    return read_check(ctx, s);
}

int dock_dof_apply(dock_ctx* ctx, int batch_id, const float* x, const float* q, int qstride, float* z, void* stream) {
    int rc = check_batch(ctx, batch_id);
    if (rc) return rc;
    const BatchH& B = ctx->batches[batch_id];
    if (!x || !q || !z) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_dof_apply: NULL buffer");
    if (qstride < 6 + B.tmax) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_dof_apply: qstride < 6 + tmax");
    CK(cudaSetDevice(ctx->device));
    ScoreParams P = score_params(ctx, B, nullptr);
    P.x = x;
    P.q = q;
    P.qstride = qstride;
    P.out = z;
    CK(launch_score(P, B.lmax, DOF_APPLY, (cudaStream_t)stream));
    return read_check(ctx, (cudaStream_t)stream);
}

int dock_dof_grad(dock_ctx* ctx, int batch_id, const float* x, const float* q, int qstride, const float* grad_z,
                  float* grad_q, void* stream) {
    int rc = check_batch(ctx, batch_id);
    if (rc) return rc;
    const BatchH& B = ctx->batches[batch_id];
    if (!x || !q || !grad_z || !grad_q) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_dof_grad: NULL buffer");
    if (qstride < 6 + B.tmax) return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_dof_grad: qstride < 6 + tmax");
    CK(cudaSetDevice(ctx->device));
    ScoreParams P = score_params(ctx, B, nullptr);
    P.x = x;
    P.q = q;
    P.qstride = qstride;
    P.grad_in = grad_z;
    P.out = grad_q;
    CK(launch_score(P, B.lmax, DOF_GRAD, (cudaStream_t)stream));
    return read_check(ctx, (cudaStream_t)stream);
}

int dock_refine(dock_ctx* ctx, int batch_id, const int32_t* pocket_ids, int npockets, const dock_knobs* k,
                const float* xyz_in, dock_result* out, float* xyz_out, int on_device, void* stream) {
    return refine_impl(ctx, batch_id, pocket_ids, npockets, k, xyz_in, out, xyz_out, on_device, nullptr,
                       (cudaStream_t)stream);
}

int dock_refine_trace(dock_ctx* ctx, int batch_id, int pocket_id, const dock_knobs* k, const float* xyz_in,
                      const dock_refine_trace_buf* tr, dock_result* out, float* xyz_out) {
    if (!tr || !tr->G || !tr->D || !tr->lam || !tr->S_new || !tr->verdict || !tr->accept || !tr->S_start ||
        !tr->S_final || !tr->status)
        return fail(ctx, DOCK_ERR_INVALID_ARG, "dock_refine_trace: NULL trace buffer");
    int32_t pid = pocket_id;
    return refine_impl(ctx, batch_id, &pid, 1, k, xyz_in, out, xyz_out, 0, tr, nullptr);
}

}  // extern "C"
