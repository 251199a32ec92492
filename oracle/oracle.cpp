// FP64 CPU oracle of the batched pose-evaluation path of GeoDock-MA
// (Gadioli et al., "Tunable Approximations to Control Time-to-Solution in an
// HPC Molecular Docking Mini-App").
//
// TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
// baseline leg of the benchmark may load this library. The CUDA path shares no
// code with it and never calls it.
//
// Everything is plain double-precision loops in the order the paper states:
//   * overlap score, Eq. 1 (Sec. 3.1), with the inner minimum over pocket
//     points tabulated on a voxel grid (field K) or computed exactly;
//   * rotamer and fragment detection (Sec. 2, Alg. 1);
//   * fragment rotation about the rotamer bond (Alg. 1);
//   * intra-ligand bump check (Alg. 1's feasibility test of the shape);
//   * greedy left-then-right sweep per rotamer with strict improvement,
//     repeated `repetitions` times, with the coarse step for fragments whose
//     relative size is at most `threshold` (Alg. 2, Sec. 3.3);
//   * tile peeling ("enable refinement", Eq. 2 and Eq. 3, Alg. 2);
//   * seeded rigid initial orientations (not in the paper).
//
// Readings where the paper is silent (each listed in the design notes):
//   - Eq. 1 sums over the l atoms and minimises over the p points (0-based,
//     exclusive bounds).
//   - Every per-atom term is floored at one voxel spacing squared (h^2), so
//     the denominator never vanishes; with the field in grid units every term
//     is then a positive integer.
//   - Maximising o = l / (h^2 S) is minimising S, the sum in grid units.
//   - Rotation angles are relative to the fragment's position at sweep start;
//     angle 0 is the incumbent and a candidate replaces the best only if its
//     score is strictly better (first maximum wins).
//   - The bump check tests every pair (i in M minus {c}, j in F minus {b}):
//     exactly the pairs whose distance changes under the torsion; a pair
//     closer than bump_thr makes the candidate infeasible.
//   - Local refinement (not in the paper; it only mentions steepest descent
//     loosely): gradient ascent of the trilinear form of Eq. 1 over 3
//     translations, 3 rotations about the centroid (exponential map) and every
//     torsion (the side away from atom 0 moves; deltas applied from the
//     deepest bond to the root), each step accepted only if S drops and the
//     pose stays bump-free (and inside the box with clip_box=1).
//   - "Pose clipping": with clip_box=1 a candidate with a moving atom outside
//     the grid box is infeasible and an initial pose with any atom outside is
//     skipped; with clip_box=0 the lookup is clamped to the box and the
//     squared distance outside the box is added.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

using V3 = std::array<double, 3>;

V3 sub(const V3& a, const V3& b) { return {a[0] - b[0], a[1] - b[1], a[2] - b[2]}; }
V3 add(const V3& a, const V3& b) { return {a[0] + b[0], a[1] + b[1], a[2] + b[2]}; }
V3 mul(const V3& a, double s) { return {a[0] * s, a[1] * s, a[2] * s}; }
double dot(const V3& a, const V3& b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
V3 cross(const V3& a, const V3& b) {
    return {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
}
double norm(const V3& a) { return std::sqrt(dot(a, a)); }

}  // namespace

extern "C" {

// Mirrors of the ctypes structures in oracle/__init__.py.
struct or_grid {
    int nx, ny, nz;
    double h;
    double origin[3];  // centre of voxel (0,0,0), Å
    double centre[3];  // pocket centre, Å (initial poses put the ligand centroid here)
    const uint16_t* K;      // floored field, nx*ny*nz, x fastest (nullable in exact mode)
    const int32_t* pts;     // probe points as voxel indices (x,y,z), for exact mode
    int npts;
};

struct or_ligands {
    int n;
    const int32_t* atom_off;
    const float* xyz;
    const int32_t* bond_off;
    const int32_t* bonds;
    const int32_t* rot_off;
    const int32_t* rot;
    int64_t id_base;
    const int64_t* ids;  // per-ligand id for the pose generator (nullable: id_base + index)
};

struct or_knobs {
    double hp_step, lp_step, threshold;
    int repetitions, n_poses, clip_box, score_mode;  // score_mode: 0 nearest, 1 trilinear, 2 exact points
    int enable_refinement;
    double bump_thr;
    uint64_t seed;
    double amb_delta;  // parity band around voxel boundaries (grid units); 0 disables the flags
    double amb_bump;   // parity band around bump_thr^2 (Å^2)
};

struct or_out {
    // per ligand
    double* best_score;
    int32_t* best_pose;
    int32_t* status;  // 0 ok, 1 every initial pose skipped
    // per (ligand, pose): index atom-independent = pose_base[b] + p
    double* pose_S;        // final S, grid units (0 when skipped)
    double* pose_init_S;   // initial S
    double* pose_init_lo;  // its interval over voxel-boundary alternatives (nullable)
    double* pose_init_hi;
    int32_t* pose_status;  // 0 ok, 1 skipped
    double* pose_xyz;      // final coordinates, Å, (atom_off[b]*N + p*l_b)*3 (nullable)
    double* init_xyz;      // initial coordinates, same layout (nullable)
    // sweep trace (all nullable); sweep index = sweep_base[b] + p*nsweep_b + s
    const int64_t* sweep_base;
    const int32_t* force_k;  // replay: commit this candidate instead of the own argmax
    int32_t* chosen_k;
    int32_t* own_k;
    int32_t pmax;            // candidate stride of the per-candidate arrays
    double* cand_S;          // S of candidate k (k = 0: incumbent)
    double* cand_lo;         // lower/upper end of S over voxel-boundary alternatives
    double* cand_hi;
    int32_t* cand_status;    // 1 feasible, 0 bump, -1 outside box, -2 no such candidate
    int32_t* cand_amb;       // bit0 score interval, bit1 bump band, bit2 box band
};

// Local refinement knobs and outputs (trilinear score, gradient ascent).
struct or_refine_knobs {
    int steps, clip_box;
    double bump_thr;
    double lambda0, lambda_max, grow, shrink;  // step length (max atom displacement, Å) and its update
    double amb_delta, amb_bump, amb_rel;       // parity bands (grid units, Å^2, relative S)
};

struct or_refine_out {
    // per ligand
    double* S_start;   // trilinear S of the start pose (grid units)
    double* S_final;
    int32_t* status;   // 0 refined, 1 skipped (start pose outside the box with clip_box=1)
    double* xyz;       // final coordinates, Å, atom_off[b]*3 (nullable)
    // per (ligand, step), index b*steps + s (all nullable)
    int32_t gstride;   // stride of G: 6 + the largest torsion count
    double* G;         // d o / d (t, omega, theta) at the step's start pose
    double* D;         // largest atom displacement per unit of G (Å)
    double* lambda;    // step length used
    double* S_new;     // S of the trial pose
    int32_t* verdict;  // bit0 S_new < S, bit1 bump-free, bit2 inside the box
    int32_t* accept;   // the committed decision
    int32_t* flags;    // bit0 |S_new - S| within amb_rel S, bit1 pair in the bump band, bit2 atom in the box band,
                       // bit3 an atom of the step's start pose within amb_delta of a cell face (one-sided gradients)
    const int32_t* force_accept;  // replay: commit these decisions instead of the own ones
    const double* force_G;        // replay: the step direction to use where bit3 is set (same layout as G)
};

}  // extern "C"

namespace {

// ---------------------------------------------------------------- field (a1)

// K(v) = min_j |v - p_j|^2 in grid units (integers), floored at 1.
// Fills nz slices starting at slice z0 into K (slice z0 first).
void build_field(int nx, int ny, int nz, const int32_t* pts, int npts, uint16_t* K, int z0 = 0) {
    for (int zz = 0; zz < nz; ++zz)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t best = INT64_MAX;
                for (int j = 0; j < npts; ++j) {
                    int z = z0 + zz;
                    int64_t dx = x - pts[3 * j], dy = y - pts[3 * j + 1], dz = z - pts[3 * j + 2];
                    int64_t d2 = dx * dx + dy * dy + dz * dz;
                    if (d2 < best) best = d2;
                }
                if (best < 1) best = 1;
                K[(int64_t(zz) * ny + y) * nx + x] = uint16_t(best);
            }
}

// ---------------------------------------------------------------- score (Eq. 1)

struct Grid {
    const or_grid* g;
    int n[3];
    uint16_t at(int x, int y, int z) const { return g->K[(int64_t(z) * n[1] + y) * n[0] + x]; }
    V3 to_grid(const V3& x) const {
        return {(x[0] - g->origin[0]) / g->h, (x[1] - g->origin[1]) / g->h, (x[2] - g->origin[2]) / g->h};
    }
};

// Per-atom term D (grid units) with its parity interval and box flags.
struct Term {
    double D, lo, hi;
    bool inbox;      // the exact position is inside the box
    bool box_amb;    // some voxel-boundary alternative disagrees on inside/outside
    bool score_amb;  // lo < hi
};

// Nearest voxel: v = floor(t + 0.5) per axis, inside iff 0 <= v < n.
Term term_nearest(const Grid& G, const V3& x, bool clip, double delta) {
    V3 t = G.to_grid(x);
    int v[3];
    double excess2 = 0.0;
    bool inside = true;
    for (int a = 0; a < 3; ++a) {
        v[a] = int(std::floor(t[a] + 0.5));
        if (v[a] < 0 || v[a] >= G.n[a]) inside = false;
        double lo_edge = -0.5, hi_edge = G.n[a] - 0.5;
        double e = t[a] < lo_edge ? lo_edge - t[a] : (t[a] > hi_edge ? t[a] - hi_edge : 0.0);
        excess2 += e * e;
    }
    auto value = [&](const int* w, bool* in) {
        int c[3];
        bool ok = true;
        for (int a = 0; a < 3; ++a) {
            if (w[a] < 0 || w[a] >= G.n[a]) ok = false;
            c[a] = std::min(std::max(w[a], 0), G.n[a] - 1);
        }
        *in = ok;
        return double(G.at(c[0], c[1], c[2]));
    };
    Term r{};
    bool in0;
    double D0 = value(v, &in0);
    r.inbox = in0;
    r.D = D0 + (in0 ? 0.0 : excess2);
    if (!in0 && clip) r.D = D0;  // value unused: the candidate is infeasible
    r.lo = r.hi = r.D;
    r.box_amb = r.score_amb = false;
    if (delta > 0.0) {
        // alternatives on each axis whose fractional position lies within delta of a rounding edge
        std::vector<int> alt[3];
        for (int a = 0; a < 3; ++a) {
            alt[a].push_back(v[a]);
            double f = t[a] + 0.5 - std::floor(t[a] + 0.5);
            if (f < delta) alt[a].push_back(v[a] - 1);
            if (f > 1.0 - delta) alt[a].push_back(v[a] + 1);
        }
        for (int i : alt[0])
            for (int j : alt[1])
                for (int k : alt[2]) {
                    int w[3] = {i, j, k};
                    bool in;
                    double D = value(w, &in);
                    if (in != in0) r.box_amb = true;
                    if (!in) {
                        if (clip) continue;
                        D += excess2;
                    }
                    r.lo = std::min(r.lo, D);
                    r.hi = std::max(r.hi, D);
                }
        r.score_amb = r.lo < r.hi;
    }
    return r;
}

// Trilinear interpolation of the floored field between voxel centres; inside
// iff 0 <= t <= n-1 on every axis.
Term term_trilinear(const Grid& G, const V3& x, bool clip, double delta) {
    V3 t = G.to_grid(x);
    double tc[3];
    double excess2 = 0.0;
    bool inside = true, amb = false;
    for (int a = 0; a < 3; ++a) {
        double hi_edge = G.n[a] - 1;
        tc[a] = std::min(std::max(t[a], 0.0), hi_edge);
        double e = t[a] - tc[a];
        excess2 += e * e;
        if (t[a] < 0.0 || t[a] > hi_edge) inside = false;
        if (delta > 0.0 && (std::fabs(t[a]) <= delta || std::fabs(t[a] - hi_edge) <= delta)) amb = true;
    }
    int i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        i0[a] = std::min(int(std::floor(tc[a])), G.n[a] - 2);
        f[a] = tc[a] - i0[a];
    }
    double D = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
                D += w * G.at(i0[0] + dx, i0[1] + dy, i0[2] + dz);
            }
    Term r{};
    r.inbox = inside;
    r.D = D + ((inside || clip) ? 0.0 : excess2);
    r.lo = r.hi = r.D;
    r.box_amb = amb;
    r.score_amb = false;
    return r;
}

// Exact point form of Eq. 1: min over the probe points of the squared
// distance, in grid units, floored at 1. Inside/outside as for nearest.
Term term_exact(const Grid& G, const V3& x, bool clip, double delta) {
    (void)clip;
    V3 t = G.to_grid(x);
    double best = INFINITY;
    for (int j = 0; j < G.g->npts; ++j) {
        double dx = t[0] - G.g->pts[3 * j], dy = t[1] - G.g->pts[3 * j + 1], dz = t[2] - G.g->pts[3 * j + 2];
        best = std::min(best, dx * dx + dy * dy + dz * dz);
    }
    Term r{};
    r.D = std::max(best, 1.0);
    r.lo = r.hi = r.D;
    bool inside = true, amb = false;
    for (int a = 0; a < 3; ++a) {
        int v = int(std::floor(t[a] + 0.5));
        if (v < 0 || v >= G.n[a]) inside = false;
        double f = t[a] + 0.5 - std::floor(t[a] + 0.5);
        if (delta > 0.0 && ((v == 0 && f < delta) || (v == G.n[a] - 1 && f > 1.0 - delta) ||
                            (v == -1 && f > 1.0 - delta) || (v == G.n[a] && f < delta)))
            amb = true;
    }
    r.inbox = inside;
    r.box_amb = amb;
    r.score_amb = false;
    return r;
}

Term term(const Grid& G, int mode, const V3& x, bool clip, double delta) {
    if (mode == 1) return term_trilinear(G, x, clip, delta);
    if (mode == 2) return term_exact(G, x, clip, delta);
    return term_nearest(G, x, clip, delta);
}

// S = sum of the per-atom terms (grid units); o = l / (h^2 S) is Eq. 1.
struct Score {
    double S, lo, hi;
    bool inbox, box_amb, score_amb;
};
Score score_all(const Grid& G, int mode, const std::vector<V3>& x, bool clip, double delta) {
    Score s{0, 0, 0, true, false, false};
    for (const V3& xi : x) {
        Term t = term(G, mode, xi, clip, delta);
        s.S += t.D;
        s.lo += t.lo;
        s.hi += t.hi;
        s.inbox = s.inbox && t.inbox;
        s.box_amb = s.box_amb || t.box_amb;
        s.score_amb = s.score_amb || t.score_amb;
    }
    return s;
}

// ---------------------------------------------------------- ligand topology

struct Mol {
    int l = 0;
    std::vector<V3> x0;
    std::vector<std::array<int, 2>> bonds;
    std::vector<int> rot;
    std::vector<std::vector<int>> adj;
};

// Atoms reachable from `start` without crossing bond `skip` (Sec. 2: removing
// a rotamer splits the ligand into two non-empty fragments).
std::vector<char> component(const Mol& m, int start, int skip) {
    std::vector<char> in(m.l, 0);
    std::vector<int> stack{start};
    in[start] = 1;
    int su = m.bonds[skip][0], sv = m.bonds[skip][1];
    while (!stack.empty()) {
        int u = stack.back();
        stack.pop_back();
        for (int v : m.adj[u]) {
            if ((u == su && v == sv) || (u == sv && v == su)) continue;
            if (!in[v]) { in[v] = 1; stack.push_back(v); }
        }
    }
    return in;
}

// One fragment sweep (Alg. 1): the moving side M, its bond atom c and the
// fixed bond atom b.
struct Side {
    std::vector<char> moving;
    int c, b, m;
};

// Left then right fragment of every rotatable bond, in the given order; the
// left fragment is the side of the lower atom index.
bool sides_of(const Mol& m, std::vector<Side>& out) {
    for (int r : m.rot) {
        int u = std::min(m.bonds[r][0], m.bonds[r][1]);
        int v = std::max(m.bonds[r][0], m.bonds[r][1]);
        std::vector<char> L = component(m, u, r);
        if (L[v]) return false;  // not a rotamer: the bond closes a ring
        std::vector<char> R(m.l);
        for (int i = 0; i < m.l; ++i) R[i] = !L[i];
        int mL = 0;
        for (char c : L) mL += c;
        out.push_back({L, u, v, mL});
        out.push_back({R, v, u, m.l - mL});
    }
    return true;
}

// ------------------------------------------------------------- rotation (Alg. 1)

// Rotate point x by theta (radians) about the axis through c with unit
// direction k, right-handed (Rodrigues' formula).
V3 rotate(const V3& x, const V3& c, const V3& k, double theta) {
    V3 v = sub(x, c);
    double ct = std::cos(theta), st = std::sin(theta);
    V3 r = add(add(mul(v, ct), mul(cross(k, v), st)), mul(k, dot(k, v) * (1.0 - ct)));
    return add(c, r);
}

// Number of candidate angles k*step (k = 0, 1, ...) below 360 degrees.
int n_angles(double step) {
    int P = int(std::ceil(360.0 / step));
    while (P > 1 && (P - 1) * step >= 360.0) --P;
    while (P * step < 360.0) ++P;
    return P;
}

// Tile size for tile peeling (Eq. 3): the divisor of 360 that is a multiple
// of the step and lies nearest to sqrt(360 * step); ties go to the smaller.
int peel_tile(double step) {
    double target = std::sqrt(360.0 * step);
    int best = -1;
    double bestd = INFINITY;
    for (int x = 1; x <= 360; ++x) {
        if (360 % x) continue;
        double q = x / step;
        if (std::fabs(q - std::round(q)) > 1e-9 || q < 1.0 - 1e-9) continue;
        double d = std::fabs(x - target);
        if (d < bestd - 1e-12) { bestd = d; best = x; }
    }
    return best;
}

// ------------------------------------------------------------ poses (not in paper)

uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
// The (ctr+1)-th output of SplitMix64 started at `seed`, as a double in [0,1).
double draw(uint64_t seed, uint64_t ctr) {
    uint64_t z = sm_mix(seed + (ctr + 1) * 0x9e3779b97f4a7c15ULL);
    return double(z >> 11) * 0x1.0p-53;
}

// Rotation of pose p: identity for p = 0, else Shoemake's uniform random
// quaternion (Graphics Gems III, 1992) from three counter-based draws.
std::array<double, 9> pose_rotation(uint64_t seed, int64_t id, int p) {
    if (p == 0) return {1, 0, 0, 0, 1, 0, 0, 0, 1};
    uint64_t base = (uint64_t(id) * 4096 + uint64_t(p)) * 4;
    double u1 = draw(seed, base), u2 = draw(seed, base + 1), u3 = draw(seed, base + 2);
    const double two_pi = 6.283185307179586476925286766559;
    double r1 = std::sqrt(1.0 - u1), r2 = std::sqrt(u1);
    double qx = r1 * std::sin(two_pi * u2), qy = r1 * std::cos(two_pi * u2);
    double qz = r2 * std::sin(two_pi * u3), qw = r2 * std::cos(two_pi * u3);
    return {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw), 2 * (qx * qz + qy * qw),
            2 * (qx * qy + qz * qw), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw),
            2 * (qx * qz - qy * qw), 2 * (qy * qz + qx * qw), 1 - 2 * (qx * qx + qy * qy)};
}

// ------------------------------------------------------------------ docking

struct Ctx {
    Grid G;
    const or_knobs* k;
    const or_ligands* L;
    or_out* o;
};

// Evaluate one candidate rotation of side s by theta; returns its score and
// status with the parity flags.
struct Cand {
    double S, lo, hi;
    int status;  // 1 feasible, 0 bump, -1 outside box
    int amb;
};

Cand evaluate(const Ctx& C, const std::vector<V3>& x, const Side& s, double theta, std::vector<V3>& y) {
    const or_knobs& K = *C.k;
    bool clip = K.clip_box != 0;
    y = x;
    V3 axis = sub(x[s.c], x[s.b]);
    axis = mul(axis, 1.0 / norm(axis));
    int n = int(x.size());
    for (int i = 0; i < n; ++i)
        if (s.moving[i] && i != s.c) y[i] = rotate(x[i], x[s.c], axis, theta);
    Cand r{0, 0, 0, 1, 0};
    // bump check over the pairs whose distance depends on this torsion
    double thr2 = K.bump_thr * K.bump_thr;
    bool clash = false;
    for (int i = 0; i < n; ++i) {
        if (!s.moving[i] || i == s.c) continue;
        for (int j = 0; j < n; ++j) {
            if (s.moving[j] || j == s.b) continue;
            V3 d = sub(y[i], x[j]);
            double d2 = dot(d, d);
            if (d2 < thr2) clash = true;
            if (K.amb_bump > 0 && std::fabs(d2 - thr2) <= K.amb_bump) r.amb |= 2;
        }
    }
    Score sc = score_all(C.G, K.score_mode, y, clip, K.amb_delta);
    r.S = sc.S;
    r.lo = sc.lo;
    r.hi = sc.hi;
    if (sc.score_amb) r.amb |= 1;
    if (sc.box_amb) r.amb |= 4;
    if (clash) r.status = 0;
    else if (clip && !sc.inbox) r.status = -1;
    return r;
}

void dock_ligand(const Ctx& C, int b) {
    const or_ligands& L = *C.L;
    const or_knobs& K = *C.k;
    or_out& O = *C.o;
    Mol m;
    int a0 = L.atom_off[b];
    m.l = L.atom_off[b + 1] - a0;
    for (int i = 0; i < m.l; ++i)
        m.x0.push_back({double(L.xyz[3 * (a0 + i)]), double(L.xyz[3 * (a0 + i) + 1]), double(L.xyz[3 * (a0 + i) + 2])});
    m.adj.assign(m.l, {});
    for (int e = L.bond_off[b]; e < L.bond_off[b + 1]; ++e) {
        int u = L.bonds[2 * e], v = L.bonds[2 * e + 1];
        m.bonds.push_back({u, v});
        m.adj[u].push_back(v);
        m.adj[v].push_back(u);
    }
    for (int r = L.rot_off[b]; r < L.rot_off[b + 1]; ++r) m.rot.push_back(L.rot[r]);
    std::vector<Side> sides;
    bool topo_ok = sides_of(m, sides);
    const int N = K.n_poses;
    const int nsweep = K.repetitions * int(sides.size());
    int64_t pose_base = int64_t(b) * N;
    const double h2 = C.G.g->h * C.G.g->h;

    V3 g{0, 0, 0};
    for (const V3& xi : m.x0) g = add(g, xi);
    g = mul(g, 1.0 / m.l);
    V3 centre{C.G.g->centre[0], C.G.g->centre[1], C.G.g->centre[2]};
    const int P_hp = n_angles(K.hp_step), P_lp = n_angles(K.lp_step);

    double best_S = INFINITY;
    int best_p = -1;
    for (int p = 0; p < N; ++p) {
        // initial rigid orientation about the centroid, centroid on the pocket centre
        std::array<double, 9> R = pose_rotation(K.seed, L.ids ? L.ids[b] : L.id_base + b, p);
        std::vector<V3> x(m.l);
        for (int i = 0; i < m.l; ++i) {
            V3 d = sub(m.x0[i], g);
            x[i] = add(centre, V3{R[0] * d[0] + R[1] * d[1] + R[2] * d[2], R[3] * d[0] + R[4] * d[1] + R[5] * d[2],
                                  R[6] * d[0] + R[7] * d[1] + R[8] * d[2]});
        }
        int64_t xo = (int64_t(a0) * N + int64_t(p) * m.l) * 3;
        if (O.init_xyz)
            for (int i = 0; i < m.l; ++i)
                for (int a = 0; a < 3; ++a) O.init_xyz[xo + 3 * i + a] = x[i][a];
        bool clip = K.clip_box != 0;
        Score s0 = score_all(C.G, K.score_mode, x, clip, K.amb_delta);
        double S_cur = s0.S;
        if (O.pose_init_S) O.pose_init_S[pose_base + p] = S_cur;
        if (O.pose_init_lo) O.pose_init_lo[pose_base + p] = s0.lo;
        if (O.pose_init_hi) O.pose_init_hi[pose_base + p] = s0.hi;
        bool skipped = !topo_ok || (clip && !s0.inbox);
        if (O.pose_status) O.pose_status[pose_base + p] = skipped ? 1 : 0;
        if (skipped) {
            if (O.pose_S) O.pose_S[pose_base + p] = 0.0;
            if (O.pose_xyz)
                for (int i = 0; i < m.l; ++i)
                    for (int a = 0; a < 3; ++a) O.pose_xyz[xo + 3 * i + a] = x[i][a];
            continue;
        }
        std::vector<V3> y;
        for (int rep = 0; rep < K.repetitions; ++rep) {
            for (size_t si = 0; si < sides.size(); ++si) {
                const Side& s = sides[si];
                int sweep = rep * int(sides.size()) + int(si);
                int64_t tix = O.sweep_base ? O.sweep_base[b] + int64_t(p) * nsweep + sweep : -1;
                // Alg. 2: coarse step for fragments of relative size <= threshold
                bool coarse = double(s.m) / double(m.l) <= K.threshold;
                double step = coarse ? K.lp_step : K.hp_step;
                int P = coarse ? P_lp : P_hp;
                // incumbent: the fragment where it is (angle 0)
                Score inc = score_all(C.G, K.score_mode, x, clip, K.amb_delta);
                auto record = [&](int kslot, const Cand& c) {
                    if (tix < 0 || !O.cand_S) return;
                    int64_t ci = tix * O.pmax + kslot;
                    O.cand_S[ci] = c.S;
                    if (O.cand_lo) O.cand_lo[ci] = c.lo;
                    if (O.cand_hi) O.cand_hi[ci] = c.hi;
                    if (O.cand_status) O.cand_status[ci] = c.status;
                    if (O.cand_amb) O.cand_amb[ci] = c.amb;
                };
                if (tix >= 0 && O.cand_S)
                    for (int k = 0; k < O.pmax; ++k) {
                        int64_t ci = tix * O.pmax + k;
                        O.cand_S[ci] = 0;
                        if (O.cand_lo) O.cand_lo[ci] = 0;
                        if (O.cand_hi) O.cand_hi[ci] = 0;
                        if (O.cand_status) O.cand_status[ci] = -2;
                        if (O.cand_amb) O.cand_amb[ci] = 0;
                    }
                Cand c0{S_cur, inc.lo, inc.hi, 1, inc.score_amb ? 1 : 0};
                record(0, c0);
                const double deg = 3.14159265358979323846 / 180.0;
                int best_k = 0;
                double best = S_cur;
                std::vector<double> thetas;  // candidate slot -> angle (degrees)
                thetas.push_back(0.0);
                if (K.enable_refinement && !coarse) {
                    // tile peeling (Alg. 2, Eq. 2-3): centre of every tile, then
                    // every step of the best tile; slots 1.. are the peels, then the tile
                    int x_t = peel_tile(step);
                    int ntile = 360 / x_t;
                    int best_tile = -1;
                    double best_peel = INFINITY;
                    for (int t = 0; t < ntile; ++t) {
                        double th = t * x_t + 0.5 * x_t;
                        thetas.push_back(th);
                        Cand c = evaluate(C, x, s, th * deg, y);
                        record(int(thetas.size()) - 1, c);
                        if (c.status == 1 && c.S < best_peel) { best_peel = c.S; best_tile = t; }
                    }
                    if (best_tile >= 0) {
                        int per = int(std::lround(x_t / step));
                        for (int j = 0; j < per; ++j) {
                            double th = best_tile * x_t + j * step;
                            thetas.push_back(th);
                            int slot = int(thetas.size()) - 1;
                            Cand c = evaluate(C, x, s, th * deg, y);
                            record(slot, c);
                            if (c.status == 1 && c.S < best) { best = c.S; best_k = slot; }
                        }
                    }
                } else {
                    for (int k = 1; k < P; ++k) {
                        double th = k * step;
                        thetas.push_back(th);
                        Cand c = evaluate(C, x, s, th * deg, y);
                        record(k, c);
                        if (c.status == 1 && c.S < best) { best = c.S; best_k = k; }
                    }
                }
                int commit = best_k;
                if (O.own_k && tix >= 0) O.own_k[tix] = best_k;
                if (O.force_k && tix >= 0) commit = O.force_k[tix];
                if (commit < 0 || commit >= int(thetas.size())) commit = best_k;  // guarded by the caller
                if (O.chosen_k && tix >= 0) O.chosen_k[tix] = commit;
                if (commit != 0) {
                    Cand c = evaluate(C, x, s, thetas[commit] * deg, y);
                    x = y;
                    S_cur = c.S;
                }
            }
        }
        if (O.pose_S) O.pose_S[pose_base + p] = S_cur;
        if (O.pose_xyz)
            for (int i = 0; i < m.l; ++i)
                for (int a = 0; a < 3; ++a) O.pose_xyz[xo + 3 * i + a] = x[i][a];
        if (S_cur < best_S) { best_S = S_cur; best_p = p; }
    }
    if (O.best_pose) O.best_pose[b] = best_p;
    if (O.status) O.status[b] = best_p < 0 ? 1 : 0;
    if (O.best_score) O.best_score[b] = best_p < 0 ? 0.0 : double(m.l) / (h2 * best_S);
}


// ------------------------------------------------ local refinement (not in the paper)

Mol load_mol(const or_ligands& L, int b, std::vector<V3>* x0 = nullptr) {
    Mol m;
    int a0 = L.atom_off[b];
    m.l = L.atom_off[b + 1] - a0;
    for (int i = 0; i < m.l; ++i)
        m.x0.push_back({double(L.xyz[3 * (a0 + i)]), double(L.xyz[3 * (a0 + i) + 1]), double(L.xyz[3 * (a0 + i) + 2])});
    m.adj.assign(m.l, {});
    for (int e = L.bond_off[b]; e < L.bond_off[b + 1]; ++e) {
        int u = L.bonds[2 * e], v = L.bonds[2 * e + 1];
        m.bonds.push_back({u, v});
        m.adj[u].push_back(v);
        m.adj[v].push_back(u);
    }
    for (int r = L.rot_off[b]; r < L.rot_off[b + 1]; ++r) m.rot.push_back(L.rot[r]);
    if (x0) *x0 = m.x0;
    return m;
}

// Trilinear term of one atom at grid position t with its gradient dD/dt
// (grid units). Outside the box the term is taken at the clamped position; with
// clip_box=0 the squared excess is added, so its gradient is 2 (t - clamp(t)).
double trilinear_grad(const Grid& G, const V3& t, bool clip, V3& dD, bool& inside) {
    double tc[3], f[3];
    int i0[3];
    bool out_axis[3];
    double excess2 = 0.0;
    inside = true;
    for (int a = 0; a < 3; ++a) {
        double hi_edge = G.n[a] - 1;
        tc[a] = std::min(std::max(t[a], 0.0), hi_edge);
        out_axis[a] = t[a] < 0.0 || t[a] > hi_edge;
        if (out_axis[a]) inside = false;
        excess2 += (t[a] - tc[a]) * (t[a] - tc[a]);
        i0[a] = std::min(int(std::floor(tc[a])), G.n[a] - 2);
        f[a] = tc[a] - i0[a];
    }
    double D = 0.0;
    dD = {0, 0, 0};
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double K = G.at(i0[0] + dx, i0[1] + dy, i0[2] + dz);
                double wx = dx ? f[0] : 1.0 - f[0], wy = dy ? f[1] : 1.0 - f[1], wz = dz ? f[2] : 1.0 - f[2];
                double sx = dx ? 1.0 : -1.0, sy = dy ? 1.0 : -1.0, sz = dz ? 1.0 : -1.0;
                D += wx * wy * wz * K;
                dD[0] += sx * wy * wz * K;
                dD[1] += wx * sy * wz * K;
                dD[2] += wx * wy * sz * K;
            }
    for (int a = 0; a < 3; ++a)
        if (out_axis[a]) dD[a] = clip ? 0.0 : 2.0 * (t[a] - tc[a]);
    if (!clip && !inside) D += excess2;
    return D;
}

// Torsion degrees of freedom: for every rotatable bond (in the ligand's order)
// the side away from atom 0 moves about the axis from b to c (c in the moving
// side). Deltas are applied from the deepest bond (depth of c from atom 0) to
// the root, ties in bond order.
struct Torsion {
    std::vector<char> M;
    int c, b, depth;
};
struct Dofs {
    std::vector<Torsion> tor;
    std::vector<int> order;
    std::vector<std::vector<char>> check;  // pairs tested by the bump check
};

Dofs dofs_of(const Mol& m) {
    Dofs d;
    std::vector<int> depth(m.l, -1);
    std::vector<int> queue{0};
    depth[0] = 0;
    for (size_t h = 0; h < queue.size(); ++h)
        for (int v : m.adj[queue[h]])
            if (depth[v] < 0) { depth[v] = depth[queue[h]] + 1; queue.push_back(v); }
    d.check.assign(m.l, std::vector<char>(m.l, 0));
    for (int r : m.rot) {
        int u = m.bonds[r][0], v = m.bonds[r][1];
        std::vector<char> root_side = component(m, 0, r);
        Torsion t;
        t.c = root_side[u] ? v : u;
        t.b = root_side[u] ? u : v;
        t.M.assign(m.l, 0);
        for (int i = 0; i < m.l; ++i) t.M[i] = !root_side[i];
        t.depth = depth[t.c];
        // the pairs whose distance this torsion changes (Alg. 1's bump pairs)
        for (int i = 0; i < m.l; ++i)
            for (int j = 0; j < m.l; ++j)
                if (t.M[i] && i != t.c && !t.M[j] && j != t.b) d.check[i][j] = d.check[j][i] = 1;
        d.tor.push_back(t);
    }
    for (int k = 0; k < int(d.tor.size()); ++k) d.order.push_back(k);
    std::stable_sort(d.order.begin(), d.order.end(), [&](int a, int b) { return d.tor[a].depth > d.tor[b].depth; });
    return d;
}

V3 centroid(const std::vector<V3>& x) {
    V3 g{0, 0, 0};
    for (const V3& xi : x) g = add(g, xi);
    return mul(g, 1.0 / double(x.size()));
}

// Rotation matrix of the rotation vector w (Rodrigues' formula).
std::array<double, 9> expmap(const V3& w) {
    double th = norm(w);
    std::array<double, 9> R{1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (th == 0.0) return R;
    V3 k = mul(w, 1.0 / th);
    double c = std::cos(th), s = std::sin(th), C = 1.0 - c;
    R = {c + k[0] * k[0] * C,        k[0] * k[1] * C - k[2] * s, k[0] * k[2] * C + k[1] * s,
         k[1] * k[0] * C + k[2] * s, c + k[1] * k[1] * C,        k[1] * k[2] * C - k[0] * s,
         k[2] * k[0] * C - k[1] * s, k[2] * k[1] * C + k[0] * s, c + k[2] * k[2] * C};
    return R;
}

// z = g + R(omega) (tau(x) - g) + t, with tau the torsion deltas and g the centroid of x.
std::vector<V3> dof_apply(const Dofs& d, const std::vector<V3>& x, const double* q) {
    std::vector<V3> y = x;
    for (int k : d.order) {
        const Torsion& t = d.tor[k];
        V3 c = y[t.c], axis = sub(y[t.c], y[t.b]);
        axis = mul(axis, 1.0 / norm(axis));
        for (size_t i = 0; i < y.size(); ++i)
            if (t.M[i] && int(i) != t.c) y[i] = rotate(y[i], c, axis, q[6 + k]);
    }
    V3 g = centroid(x);
    std::array<double, 9> R = expmap({q[3], q[4], q[5]});
    std::vector<V3> z(y.size());
    for (size_t i = 0; i < y.size(); ++i) {
        V3 v = sub(y[i], g);
        z[i] = add(add(g, {R[0] * v[0] + R[1] * v[1] + R[2] * v[2], R[3] * v[0] + R[4] * v[1] + R[5] * v[2],
                           R[6] * v[0] + R[7] * v[1] + R[8] * v[2]}),
                   {q[0], q[1], q[2]});
    }
    return z;
}

// d f / d q from p_i = d f / d z_i at the pose z = dof_apply(x, q):
//   translation: sum_i p_i;
//   rotation: J(omega)^T sum_i (z_i - g - t) x p_i, J the left Jacobian of the
//     exponential map, I + (1 - cos a)/a^2 [w]x + (a - sin a)/a^3 [w]x^2 (a = |w|);
//   torsion k: axis_k . sum_{i in M_k} (z_i - z_c) x p_i, with the axis and c
//     taken in z (a later rigid motion of bond k's side carries its axis along).
void dof_grad(const Dofs& d, const std::vector<V3>& x, const double* q, const std::vector<V3>& z,
              const std::vector<V3>& p, double* G) {
    V3 g = centroid(x), t{q[0], q[1], q[2]}, w{q[3], q[4], q[5]};
    V3 gt{0, 0, 0}, tau{0, 0, 0};
    for (size_t i = 0; i < z.size(); ++i) {
        gt = add(gt, p[i]);
        tau = add(tau, cross(sub(sub(z[i], g), t), p[i]));
    }
    double a = norm(w), A, B;
    if (a < 1e-4) {
        A = 0.5 - a * a / 24.0;
        B = 1.0 / 6.0 - a * a / 120.0;
    } else {
        A = (1.0 - std::cos(a)) / (a * a);
        B = (a - std::sin(a)) / (a * a * a);
    }
    // J^T v = v - A (w x v) + B (w x (w x v))   ([w]x^T = -[w]x)
    V3 wv = cross(w, tau), wwv = cross(w, wv);
    V3 gw = add(sub(tau, mul(wv, A)), mul(wwv, B));
    for (int a3 = 0; a3 < 3; ++a3) {
        G[a3] = gt[a3];
        G[3 + a3] = gw[a3];
    }
    for (size_t k = 0; k < d.tor.size(); ++k) {
        const Torsion& tk = d.tor[k];
        V3 axis = sub(z[tk.c], z[tk.b]);
        axis = mul(axis, 1.0 / norm(axis));
        V3 s{0, 0, 0};
        for (size_t i = 0; i < z.size(); ++i)
            if (tk.M[i]) s = add(s, cross(sub(z[i], z[tk.c]), p[i]));
        G[6 + k] = dot(axis, s);
    }
}

// Trilinear S of a pose with dS/dz (grid units per Å) and the box flags.
double score_grad(const Grid& G, const std::vector<V3>& z, bool clip, double delta, std::vector<V3>* dS, bool& inside,
                  bool& box_amb) {
    double S = 0.0;
    inside = true;
    box_amb = false;
    if (dS) dS->assign(z.size(), {0, 0, 0});
    for (size_t i = 0; i < z.size(); ++i) {
        V3 t = G.to_grid(z[i]);
        V3 dD;
        bool in;
        S += trilinear_grad(G, t, clip, dD, in);
        inside = inside && in;
        for (int a = 0; a < 3; ++a)
            if (delta > 0.0 && (std::fabs(t[a]) <= delta || std::fabs(t[a] - (G.n[a] - 1)) <= delta)) box_amb = true;
        if (dS) (*dS)[i] = mul(dD, 1.0 / G.g->h);
    }
    return S;
}

void refine_ligand(const Grid& G, const or_ligands& L, const or_refine_knobs& K, const double* xyz_in,
                   or_refine_out& O, int b) {
    Mol m = load_mol(L, b);
    Dofs d = dofs_of(m);
    const int a0 = L.atom_off[b];
    const bool clip = K.clip_box != 0;
    const double h2 = G.g->h * G.g->h, thr2 = K.bump_thr * K.bump_thr;
    const int T = int(d.tor.size());
    std::vector<V3> z(m.l);
    for (int i = 0; i < m.l; ++i) z[i] = {xyz_in[3 * (a0 + i)], xyz_in[3 * (a0 + i) + 1], xyz_in[3 * (a0 + i) + 2]};
    bool inside, box_amb;
    std::vector<V3> dS;
    double S = score_grad(G, z, clip, 0.0, nullptr, inside, box_amb);
    if (O.S_start) O.S_start[b] = S;
    const bool skip = clip && !inside;
    if (O.status) O.status[b] = skip ? 1 : 0;
    double lambda = K.lambda0;
    std::vector<double> Gq(6 + T), q(6 + T);
    for (int st = 0; st < K.steps && !skip; ++st) {
        const int64_t si = int64_t(b) * K.steps + st;
        score_grad(G, z, clip, 0.0, &dS, inside, box_amb);
        // o = l / (h^2 S): d o / d z_i = -l / (h^2 S^2) dS/dz_i
        std::vector<V3> p(m.l);
        for (int i = 0; i < m.l; ++i) p[i] = mul(dS[i], -double(m.l) / (h2 * S * S));
        std::vector<double> zero(6 + T, 0.0);
        dof_grad(d, z, zero.data(), z, p, Gq.data());
        // the trilinear gradient is one-sided on a cell face: either side is a valid gradient
        int flags = 0;
        for (int i = 0; i < m.l && K.amb_delta > 0; ++i) {
            V3 t = G.to_grid(z[i]);
            for (int a = 0; a < 3; ++a)
                if (std::fabs(t[a] - std::round(t[a])) <= K.amb_delta) flags |= 8;
        }
        if (O.G)
            for (int k = 0; k < 6 + T; ++k) O.G[si * O.gstride + k] = Gq[k];
        if ((flags & 8) && O.force_G)
            for (int k = 0; k < 6 + T; ++k) Gq[k] = O.force_G[si * O.gstride + k];
        // largest first-order atom displacement per unit of G
        V3 g = centroid(z);
        double D = 0.0;
        for (int i = 0; i < m.l; ++i) {
            V3 di = add({Gq[0], Gq[1], Gq[2]}, cross({Gq[3], Gq[4], Gq[5]}, sub(z[i], g)));
            for (int k = 0; k < T; ++k) {
                const Torsion& tk = d.tor[k];
                if (!tk.M[i]) continue;
                V3 axis = sub(z[tk.c], z[tk.b]);
                axis = mul(axis, 1.0 / norm(axis));
                di = add(di, mul(cross(axis, sub(z[i], z[tk.c])), Gq[6 + k]));
            }
            D = std::max(D, norm(di));
        }
        if (O.D) O.D[si] = D;
        if (O.lambda) O.lambda[si] = lambda;
        int verdict = 0;
        double S_new = S;
        std::vector<V3> zn;
        if (D > 0.0) {
            for (int k = 0; k < 6 + T; ++k) q[k] = Gq[k] * (lambda / D);
            zn = dof_apply(d, z, q.data());
            bool in_new;
            S_new = score_grad(G, zn, clip, K.amb_delta, nullptr, in_new, box_amb);
            bool clash = false;
            for (int i = 0; i < m.l; ++i)
                for (int j = i + 1; j < m.l; ++j) {
                    if (!d.check[i][j]) continue;
                    V3 dv = sub(zn[i], zn[j]);
                    double d2 = dot(dv, dv);
                    if (d2 < thr2) clash = true;
                    if (K.amb_bump > 0 && std::fabs(d2 - thr2) <= K.amb_bump) flags |= 2;
                }
            if (S_new < S) verdict |= 1;
            if (!clash) verdict |= 2;
            if (in_new) verdict |= 4;
            if (K.amb_rel > 0 && std::fabs(S_new - S) <= K.amb_rel * S) flags |= 1;
            if (box_amb) flags |= 4;
        }
        int acc = (verdict & 1) && (verdict & 2) && (!clip || (verdict & 4));
        if (O.force_accept) acc = O.force_accept[si] && D > 0.0;
        if (O.S_new) O.S_new[si] = S_new;
        if (O.verdict) O.verdict[si] = verdict;
        if (O.accept) O.accept[si] = acc;
        if (O.flags) O.flags[si] = flags;
        if (acc) {
            z = zn;
            S = S_new;
            lambda = std::min(lambda * K.grow, K.lambda_max);
        } else {
            lambda *= K.shrink;
        }
    }
    if (O.S_final) O.S_final[b] = S;
    if (O.xyz)
        for (int i = 0; i < m.l; ++i)
            for (int a = 0; a < 3; ++a) O.xyz[3 * (a0 + i) + a] = z[i][a];
}

}  // namespace

extern "C" {

int oracle_field(int nx, int ny, int nz, const int32_t* pts, int npts, uint16_t* K, int nthreads) {
    if (nx < 2 || ny < 2 || nz < 2 || npts < 1) return -1;
    // each thread fills whole z-slices; the slices are independent
    if (nthreads < 1) nthreads = 1;
    std::atomic<int> next{0};
    int64_t slice = int64_t(nx) * ny;
    auto worker = [&]() {
        for (int z = next++; z < nz; z = next++) build_field(nx, ny, 1, pts, npts, K + slice * z, z);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nthreads; ++t) pool.emplace_back(worker);
    worker();
    for (auto& t : pool) t.join();
    return 0;
}

// The (ctr+1)-th raw output of SplitMix64 seeded with `seed`.
uint64_t oracle_splitmix(uint64_t seed, uint64_t ctr) { return sm_mix(seed + (ctr + 1) * 0x9e3779b97f4a7c15ULL); }

// S and the inside flag of one conformation (grid units), for hand checks.
int oracle_score(const or_grid* g, int mode, int clip, const double* xyz, int natoms, double* S, int* inside) {
    Grid G{g, {g->nx, g->ny, g->nz}};
    std::vector<V3> x(natoms);
    for (int i = 0; i < natoms; ++i) x[i] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
    Score s = score_all(G, mode, x, clip != 0, 0.0);
    *S = s.S;
    *inside = s.inbox ? 1 : 0;
    return 0;
}

// One atom's term of Eq. 1 (grid units) in score mode `mode` with its parity
// band: out3 = (D, lo, hi), the term and the ends of its interval over the
// voxel-boundary alternatives within `delta` grid units (nearest mode);
// flags bit0 inside the box, bit1 some alternative disagrees on inside/outside
// (the box band), bit2 lo < hi. For hand checks of the parity bands.
int oracle_term(const or_grid* g, int mode, int clip, const double* x, double delta, double* out3, int* flags) {
    Grid G{g, {g->nx, g->ny, g->nz}};
    Term t = term(G, mode, V3{x[0], x[1], x[2]}, clip != 0, delta);
    out3[0] = t.D;
    out3[1] = t.lo;
    out3[2] = t.hi;
    *flags = (t.inbox ? 1 : 0) | (t.box_amb ? 2 : 0) | (t.score_amb ? 4 : 0);
    return 0;
}

// Rodrigues rotation of natoms points about the axis through c along k (unit
// vector computed here) by theta radians.
void oracle_rotate(const double* xyz, int natoms, const double* c, const double* b, double theta, double* out) {
    V3 C{c[0], c[1], c[2]}, B{b[0], b[1], b[2]};
    V3 k = sub(C, B);
    k = mul(k, 1.0 / norm(k));
    for (int i = 0; i < natoms; ++i) {
        V3 r = rotate({xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]}, C, k, theta);
        for (int a = 0; a < 3; ++a) out[3 * i + a] = r[a];
    }
}

int oracle_n_angles(double step) { return n_angles(step); }
int oracle_peel_tile(double step) { return peel_tile(step); }

void oracle_pose_rotation(uint64_t seed, int64_t id, int p, double* R) {
    std::array<double, 9> r = pose_rotation(seed, id, p);
    for (int i = 0; i < 9; ++i) R[i] = r[i];
}

int oracle_dock(const or_grid* g, const or_ligands* L, const or_knobs* k, or_out* o, int nthreads) {
    if (k->n_poses < 1 || k->n_poses > 4096 || k->repetitions < 0) return -1;
    if (!(k->hp_step >= 1.0 && k->hp_step <= 360.0 && k->lp_step >= 1.0 && k->lp_step <= 360.0)) return -1;
    Ctx C{Grid{g, {g->nx, g->ny, g->nz}}, k, L, o};
    if (nthreads < 1) nthreads = 1;
    std::atomic<int> next{0};
    auto worker = [&]() {
        for (int b = next++; b < L->n; b = next++) dock_ligand(C, b);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nthreads; ++t) pool.emplace_back(worker);
    worker();
    for (auto& t : pool) t.join();
    return 0;
}

// Trilinear S (grid units), dS/dx (grid units per Å) and the inside flag of one conformation.
int oracle_trilinear_grad(const or_grid* g, int clip, const double* xyz, int natoms, double* S, double* dSdx,
                          int* inside) {
    Grid G{g, {g->nx, g->ny, g->nz}};
    std::vector<V3> z(natoms), dS;
    for (int i = 0; i < natoms; ++i) z[i] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
    bool in, amb;
    *S = score_grad(G, z, clip != 0, 0.0, &dS, in, amb);
    for (int i = 0; i < natoms; ++i)
        for (int a = 0; a < 3; ++a) dSdx[3 * i + a] = dS[i][a];
    *inside = in ? 1 : 0;
    return 0;
}

// Torsion layout of ligand b: per rotatable bond (ligand order) c, b, depth and
// the moving mask (l entries each); order = application order. Returns T or -1.
int oracle_torsions(const or_ligands* L, int b, int32_t* c, int32_t* bb, int32_t* depth, uint8_t* mask,
                    int32_t* order, uint8_t* check) {
    Mol m = load_mol(*L, b);
    std::vector<Side> sides;
    if (!sides_of(m, sides)) return -1;
    Dofs d = dofs_of(m);
    for (size_t k = 0; k < d.tor.size(); ++k) {
        c[k] = d.tor[k].c;
        bb[k] = d.tor[k].b;
        depth[k] = d.tor[k].depth;
        for (int i = 0; i < m.l; ++i) mask[k * m.l + i] = uint8_t(d.tor[k].M[i]);
        order[k] = d.order[k];
    }
    if (check)
        for (int i = 0; i < m.l; ++i)
            for (int j = 0; j < m.l; ++j) check[i * m.l + j] = uint8_t(d.check[i][j]);
    return int(d.tor.size());
}

// z = dof_apply(x, q) for ligand b (x: l x 3 Å, q: 6 + T).
int oracle_dof_apply(const or_ligands* L, int b, const double* x, const double* q, double* z) {
    Mol m = load_mol(*L, b);
    std::vector<Side> sides;
    if (!sides_of(m, sides)) return -1;
    Dofs d = dofs_of(m);
    std::vector<V3> xv(m.l);
    for (int i = 0; i < m.l; ++i) xv[i] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
    std::vector<V3> zv = dof_apply(d, xv, q);
    for (int i = 0; i < m.l; ++i)
        for (int a = 0; a < 3; ++a) z[3 * i + a] = zv[i][a];
    return 0;
}

// d f / d q of ligand b from p = d f / d z at z = dof_apply(x, q).
int oracle_dof_grad(const or_ligands* L, int b, const double* x, const double* q, const double* p, double* G) {
    Mol m = load_mol(*L, b);
    std::vector<Side> sides;
    if (!sides_of(m, sides)) return -1;
    Dofs d = dofs_of(m);
    std::vector<V3> xv(m.l), pv(m.l);
    for (int i = 0; i < m.l; ++i) {
        xv[i] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]};
        pv[i] = {p[3 * i], p[3 * i + 1], p[3 * i + 2]};
    }
    std::vector<V3> zv = dof_apply(d, xv, q);
    dof_grad(d, xv, q, zv, pv, G);
    return 0;
}

// Local refinement of every ligand of the batch from the start poses xyz_in
// (Å, atom_off layout), trilinear score.
int oracle_refine(const or_grid* g, const or_ligands* L, const or_refine_knobs* k, const double* xyz_in,
                  or_refine_out* o, int nthreads) {
    if (k->steps < 0 || !(k->lambda0 > 0) || !(k->bump_thr >= 0)) return -1;
    Grid G{g, {g->nx, g->ny, g->nz}};
    if (nthreads < 1) nthreads = 1;
    std::atomic<int> next{0};
    auto worker = [&]() {
        for (int b = next++; b < L->n; b = next++) refine_ligand(G, *L, *k, xyz_in, *o, b);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < nthreads; ++t) pool.emplace_back(worker);
    worker();
    for (auto& t : pool) t.join();
    return 0;
}

}  // extern "C"
