/*
 * Seeded synthetic inputs shaped like a virtual-screening campaign: tree-shaped
 * heavy-atom ligands with marked rotatable bonds, and noisy-ellipsoid pockets
 * given as a set of probe points on voxel centres.
 *
 * This module only draws inputs. It computes no score, no field, no rotation
 * of a fragment and no sweep: both the CUDA path and the CPU oracle take its
 * output as plain arrays.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014). Each ligand draws from its
 * own stream keyed by (seed, ligand id), so a ligand does not depend on which
 * batch or shard it is generated in.
 *
 * Build with -ffp-contract=off so x86-64 and aarch64 hosts round alike.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define SYN_PI 3.14159265358979323846

typedef struct { uint64_t s; } rng_t;

static uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
static uint64_t rng_next(rng_t* r) {
    r->s += 0x9e3779b97f4a7c15ULL;
    return sm_mix(r->s);
}
/* uniform in [0, 1) with 53 random bits */
static double rng_unif(rng_t* r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }
static double rng_range(rng_t* r, double a, double b) { return a + (b - a) * rng_unif(r); }
/* Box-Muller, one variate per call */
static double rng_normal(rng_t* r) {
    double u1 = 1.0 - rng_unif(r); /* (0, 1] */
    double u2 = rng_unif(r);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * SYN_PI * u2);
}
static int rng_int(rng_t* r, int lo, int hi) { /* inclusive */
    uint64_t span = (uint64_t)(hi - lo + 1);
    return lo + (int)(rng_next(r) % span);
}
static int rng_poisson(rng_t* r, double lam) { /* Knuth's product method */
    double L = exp(-lam), p = 1.0;
    int k = 0;
    do { k++; p *= rng_unif(r); } while (p > L);
    return k - 1;
}
static rng_t stream(uint64_t seed, int64_t id, uint64_t salt) {
    rng_t r;
    r.s = sm_mix(seed ^ sm_mix((uint64_t)id * 0x632be59bd9b4e019ULL + salt));
    return r;
}

/* ---------------------------------------------------------------- sizes */

/* kind 0: l ~ U{a0..a1}, T ~ U{b0..b1}
 * kind 1: l = clip(round(lognormal(ln a0, a1)), b0, b1), T = clip(Poisson(c0), 0, c1) */
void synth_sizes(uint64_t seed, int64_t id, int kind, const double* prm, int* l_out, int* t_out) {
    rng_t r = stream(seed, id, 0x5157u);
    if (kind == 0) {
        *l_out = rng_int(&r, (int)prm[0], (int)prm[1]);
        *t_out = rng_int(&r, (int)prm[2], (int)prm[3]);
    } else {
        double v = exp(log(prm[0]) + prm[1] * rng_normal(&r));
        int l = (int)floor(v + 0.5);
        if (l < (int)prm[2]) l = (int)prm[2];
        if (l > (int)prm[3]) l = (int)prm[3];
        int t = rng_poisson(&r, prm[4]);
        if (t > (int)prm[5]) t = (int)prm[5];
        *l_out = l;
        *t_out = t;
    }
}

/* -------------------------------------------------------------- ligands */

static void unit(double* v) {
    double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= n; v[1] /= n; v[2] /= n;
}
/* orthonormal pair perpendicular to unit e */
static void perp_basis(const double* e, double* f1, double* f2) {
    double t[3] = {1.0, 0.0, 0.0};
    if (fabs(e[0]) > 0.8) { t[0] = 0.0; t[1] = 1.0; }
    double d = t[0] * e[0] + t[1] * e[1] + t[2] * e[2];
    f1[0] = t[0] - d * e[0]; f1[1] = t[1] - d * e[1]; f1[2] = t[2] - d * e[2];
    unit(f1);
    f2[0] = e[1] * f1[2] - e[2] * f1[1];
    f2[1] = e[2] * f1[0] - e[0] * f1[2];
    f2[2] = e[0] * f1[1] - e[1] * f1[0];
}

#define SYN_MAXL 256

/* Grow one tree-shaped ligand.
 *   l atoms (2..256), T requested rotatable bonds.
 *   xyz[3l] Å, bonds[2(l-1)] (parent, child) with child = bond index + 1,
 *   rot[*] ascending bond indices (at most T), *t_out = their count.
 * Geometry: bond length U(1.3, 1.6) Å; a child sits at 109.5 ± 5 degrees from
 * its parent's own bond, siblings on tetrahedral azimuth slots 120 degrees
 * apart from a random starting dihedral. A placement is redrawn (random
 * dihedral) while it comes closer than 2.0 Å to an atom three or more bonds
 * away, or closer than 1.9 Å to an atom two bonds away; after 100 failures
 * the parent is redrawn, and after 30 parents the whole ligand is regrown. Rotatable bonds are drawn without replacement
 * among bonds whose two ends both have another neighbour. Returns 0, or -1 on
 * bad arguments, -2 if no clash-free tree was found. */
int synth_ligand(uint64_t seed, int64_t id, int l, int T, double* xyz, int* bonds, int* rot, int* t_out) {
    if (l < 2 || l > SYN_MAXL || T < 0) return -1;
    rng_t r = stream(seed, id, 0x11u);
    int parent[SYN_MAXL], deg[SYN_MAXL], nchild[SYN_MAXL], first_child[SYN_MAXL];
    double phi0[SYN_MAXL];
    int dist[SYN_MAXL], queue[SYN_MAXL];
    for (int attempt = 0; attempt < 64; ++attempt) {
        int ok = 1;
        for (int i = 0; i < l; ++i) { parent[i] = -1; deg[i] = 0; nchild[i] = 0; first_child[i] = -1; }
        xyz[0] = xyz[1] = xyz[2] = 0.0;
        for (int i = 1; i < l && ok; ++i) {
            int placed = 0, p = -1;
            /* parent: uniform among earlier atoms with degree < 4, redrawn
             * when no clash-free placement exists next to it */
            for (int pdraw = 0; pdraw < 30 && !placed; ++pdraw) {
                int cand[SYN_MAXL], nc = 0;
                for (int j = 0; j < i; ++j) if (deg[j] < 4) cand[nc++] = j;
                p = cand[rng_int(&r, 0, nc - 1)];
                /* graph distance from p to every earlier atom */
                for (int j = 0; j < i; ++j) dist[j] = -1;
                int qh = 0, qt = 0;
                dist[p] = 0; queue[qt++] = p;
                while (qh < qt) {
                    int u = queue[qh++];
                    for (int v = 0; v < i; ++v) {
                        int adj = (parent[v] == u) || (parent[u] == v);
                        if (adj && dist[v] < 0) { dist[v] = dist[u] + 1; queue[qt++] = v; }
                    }
                }
                if (nchild[p] == 0) phi0[p] = rng_range(&r, 0.0, 2.0 * SYN_PI);
                for (int tries = 0; tries < 100 && !placed; ++tries) {
                    double len = rng_range(&r, 1.3, 1.6);
                    double dir[3];
                    const double* P = xyz + 3 * p;
                    int ref = parent[p] >= 0 ? parent[p] : first_child[p];
                    if (ref < 0) { /* first bond of the root: any direction */
                        double z = rng_range(&r, -1.0, 1.0), az = rng_range(&r, 0.0, 2.0 * SYN_PI);
                        double s = sqrt(1.0 - z * z);
                        dir[0] = s * cos(az); dir[1] = s * sin(az); dir[2] = z;
                    } else {
                        double e[3] = {xyz[3 * ref] - P[0], xyz[3 * ref + 1] - P[1], xyz[3 * ref + 2] - P[2]};
                        unit(e);
                        double f1[3], f2[3];
                        perp_basis(e, f1, f2);
                        int slot = parent[p] >= 0 ? nchild[p] : nchild[p] - 1;
                        double alpha = (109.5 + rng_range(&r, -5.0, 5.0)) * SYN_PI / 180.0;
                        double phi = tries == 0 ? phi0[p] + slot * 2.0 * SYN_PI / 3.0 +
                                                      rng_range(&r, -5.0, 5.0) * SYN_PI / 180.0
                                                : rng_range(&r, 0.0, 2.0 * SYN_PI);
                        for (int a = 0; a < 3; ++a)
                            dir[a] = cos(alpha) * e[a] + sin(alpha) * (cos(phi) * f1[a] + sin(phi) * f2[a]);
                    }
                    double X[3] = {P[0] + len * dir[0], P[1] + len * dir[1], P[2] + len * dir[2]};
                    int clash = 0;
                    for (int j = 0; j < i && !clash; ++j) {
                        int gd = dist[j] + 1; /* bonds between the new atom and j */
                        if (gd < 2) continue;
                        double dx = X[0] - xyz[3 * j], dy = X[1] - xyz[3 * j + 1], dz = X[2] - xyz[3 * j + 2];
                        double d2 = dx * dx + dy * dy + dz * dz;
                        double lim = gd >= 3 ? 2.0 : 1.9;
                        if (d2 < lim * lim) clash = 1;
                    }
                    if (!clash) {
                        xyz[3 * i] = X[0]; xyz[3 * i + 1] = X[1]; xyz[3 * i + 2] = X[2];
                        placed = 1;
                    }
                }
            }
            if (!placed) { ok = 0; break; }
            parent[i] = p;
            deg[p]++; deg[i]++;
            if (first_child[p] < 0) first_child[p] = i;
            nchild[p]++;
        }
        if (!ok) continue;
        for (int i = 1; i < l; ++i) { bonds[2 * (i - 1)] = parent[i]; bonds[2 * (i - 1) + 1] = i; }
        /* rotatable: internal bonds, drawn without replacement, reported ascending */
        int inner[SYN_MAXL], ni = 0;
        for (int b = 0; b < l - 1; ++b)
            if (deg[bonds[2 * b]] >= 2 && deg[bonds[2 * b + 1]] >= 2) inner[ni++] = b;
        int t = T < ni ? T : ni;
        for (int k = 0; k < t; ++k) { /* partial Fisher-Yates */
            int j = rng_int(&r, k, ni - 1);
            int tmp = inner[k]; inner[k] = inner[j]; inner[j] = tmp;
        }
        for (int a = 1; a < t; ++a) { /* insertion sort of the chosen prefix */
            int v = inner[a], b = a - 1;
            while (b >= 0 && inner[b] > v) { inner[b + 1] = inner[b]; --b; }
            inner[b + 1] = v;
        }
        for (int k = 0; k < t; ++k) rot[k] = inner[k];
        *t_out = t;
        return 0;
    }
    return -2;
}

/* --------------------------------------------------------------- pockets */

/* Noisy ellipsoidal cavity in an n^3 grid of spacing h centred on (0,0,0).
 * Semi-axes (a, b, c) Å; radial noise N(0, sigma^2) drawn on an 18 x 36
 * (polar, azimuth) lattice and interpolated bilinearly. A voxel belongs to
 * the cavity iff its centre lies within the noisy surface. The probe points
 * are the cavity voxels whose three indices are multiples of `stride`.
 * Outputs: pts[3*cap] voxel indices (x, y, z), *npts, origin[3] = centre of
 * voxel (0,0,0) in Å, centre[3] = centroid of the probe points in Å.
 * Returns 0, or -1 if cap is too small. */
int synth_pocket(uint64_t seed, int n, double h, double a, double b, double c, double sigma, int stride,
                 int* pts, int cap, int* npts, double* origin, double* centre) {
    rng_t r = stream(seed, 0, 0x90c3u);
    enum { NT = 18, NP = 36 };
    double noise[NT][NP];
    for (int i = 0; i < NT; ++i)
        for (int j = 0; j < NP; ++j) noise[i][j] = sigma * rng_normal(&r);
    double o = -h * (n - 1) / 2.0;
    origin[0] = origin[1] = origin[2] = o;
    int cnt = 0;
    double sx = 0, sy = 0, sz = 0;
    for (int k = 0; k < n; k += stride)
        for (int j = 0; j < n; j += stride)
            for (int i = 0; i < n; i += stride) {
                double x = o + h * i, y = o + h * j, z = o + h * k;
                double rr = sqrt(x * x + y * y + z * z);
                int inside;
                if (rr == 0.0) {
                    inside = 1;
                } else {
                    double dx = x / rr, dy = y / rr, dz = z / rr;
                    double rell = 1.0 / sqrt((dx / a) * (dx / a) + (dy / b) * (dy / b) + (dz / c) * (dz / c));
                    double th = acos(dz < -1.0 ? -1.0 : (dz > 1.0 ? 1.0 : dz));
                    double ph = atan2(dy, dx);
                    if (ph < 0) ph += 2.0 * SYN_PI;
                    double ti = th / SYN_PI * (NT - 1), pj = ph / (2.0 * SYN_PI) * NP;
                    int i0 = (int)floor(ti), j0 = (int)floor(pj);
                    if (i0 >= NT - 1) i0 = NT - 2;
                    double ft = ti - i0, fp = pj - j0;
                    int j1 = (j0 + 1) % NP;
                    j0 %= NP;
                    double nz = (1 - ft) * ((1 - fp) * noise[i0][j0] + fp * noise[i0][j1]) +
                                ft * ((1 - fp) * noise[i0 + 1][j0] + fp * noise[i0 + 1][j1]);
                    inside = rr <= rell + nz;
                }
                if (!inside) continue;
                if (cnt >= cap) return -1;
                pts[3 * cnt] = i; pts[3 * cnt + 1] = j; pts[3 * cnt + 2] = k;
                sx += x; sy += y; sz += z;
                ++cnt;
            }
    *npts = cnt;
    if (cnt > 0) { centre[0] = sx / cnt; centre[1] = sy / cnt; centre[2] = sz / cnt; }
    else { centre[0] = centre[1] = centre[2] = 0.0; }
    return 0;
}

/* Uniform draws for one pocket's semi-axes (multi-pocket screening): three
 * values in U(lo, hi), sorted descending. */
void synth_semi_axes(uint64_t seed, int64_t id, double lo, double hi, double* abc) {
    rng_t r = stream(seed, id, 0xa4e5u);
    double v[3];
    for (int i = 0; i < 3; ++i) v[i] = rng_range(&r, lo, hi);
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (v[j] > v[i]) { double t = v[i]; v[i] = v[j]; v[j] = t; }
    memcpy(abc, v, sizeof v);
}

/* ----------------------------------------------------------------- batch */

void synth_batch_sizes(uint64_t seed, int64_t id0, int n, int kind, const double* prm, int* l, int* t) {
    for (int i = 0; i < n; ++i) synth_sizes(seed, id0 + i, kind, prm, &l[i], &t[i]);
}

/* Fill a CSR batch of n ligands of sizes l[i] and requested rotatable counts
 * t[i] (ids id0 + i). atom_off/bond_off/rot_off have n+1 entries; xyz holds
 * 3*sum(l) doubles, bonds 2*sum(l-1) ints, rot up to sum(t) ints (local bond
 * indices). Returns 0, or the negative code of the first ligand that failed. */
int synth_batch(uint64_t seed, int64_t id0, int n, const int* l, const int* t, int* atom_off, int* bond_off,
                int* rot_off, double* xyz, int* bonds, int* rot) {
    atom_off[0] = bond_off[0] = rot_off[0] = 0;
    for (int i = 0; i < n; ++i) {
        int got = 0;
        int rc = synth_ligand(seed, id0 + i, l[i], t[i], xyz + 3 * atom_off[i], bonds + 2 * bond_off[i],
                              rot + rot_off[i], &got);
        if (rc != 0) return rc;
        atom_off[i + 1] = atom_off[i] + l[i];
        bond_off[i + 1] = bond_off[i] + l[i] - 1;
        rot_off[i + 1] = rot_off[i] + got;
    }
    return 0;
}
