/*
 * geodock.h - C ABI of the GB300 batched pose evaluator for the geometric
 * docking kernel of GeoDock-MA (Gadioli et al., "Tunable Approximations to
 * Control Time-to-Solution in an HPC Molecular Docking Mini-App").
 *
 * For every (pocket, ligand, initial pose) the library runs the greedy
 * torsion sweep of Alg. 1/Alg. 2: for each rotamer, the left and then the
 * right fragment is rotated through its candidate angles, every candidate is
 * checked for internal bumps and scored with the overlap score of Eq. 1, and
 * the fragment is set to the best angle found. The knobs of Sec. 3.3
 * (high/low precision step, threshold, repetitions, tile peeling) are run-time
 * parameters, as are the number of seeded rigid initial orientations and pose
 * clipping. All work runs in CUDA kernels for sm_103a; there is no CPU path.
 *
 * Conventions
 *  - Every call returns 0 (DOCK_OK) or a negative DOCK_ERR_* code; the text of
 *    the last error of a context is returned by dock_last_error().
 *  - The library copies every input it is given and keeps no caller pointer.
 *  - Outputs go to caller-owned buffers. Host buffers are written before the
 *    call returns; device buffers are written in stream order on `stream`.
 *  - A context is thread-compatible, not thread-safe: one thread at a time.
 *  - Per-pair status flags (e.g. "every initial pose was outside the box")
 *    are results, not errors.
 *  - The same ABI is also built as a checked library (GEODOCK_CHECKED): its
 *    kernels test every index they derive from their inputs, and a call
 *    whose kernels found a bad one returns DOCK_ERR_CUDA with the check's
 *    code and index in dock_last_error() (the call then waits for its work).
 *    It is a debugging aid; results are otherwise those of the library.
 *
 * Units: coordinates in Å, angles in degrees. Internally the path works in
 * grid units of the pocket (Å / h) in FP32; grid values are exact integers.
 */
#ifndef GEODOCK_H
#define GEODOCK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DOCK_OK 0
#define DOCK_ERR_INVALID_ARG (-1)   /* a size, pointer, index or knob out of range */
#define DOCK_ERR_TOPOLOGY (-2)      /* a rotatable bond does not split its ligand in two */
#define DOCK_ERR_OUT_OF_MEMORY (-3) /* a device allocation failed */
#define DOCK_ERR_CUDA (-4)          /* a CUDA runtime call failed (text in dock_last_error) */
#define DOCK_ERR_TIMEOUT (-5)       /* reserved for a bounded device-side wait that gives up; no kernel of this
                                       library waits on a flag (its work queue is one atomic counter), so no
                                       call returns it */
#define DOCK_ERR_UNSUPPORTED (-6)   /* a knob combination the library does not run */

/* largest ligand (atoms) and the largest grid edge (voxels) */
#define DOCK_MAX_ATOMS 255
#define DOCK_MAX_GRID 256
#define DOCK_MAX_POSES 4096

typedef struct dock_ctx dock_ctx;

/* A pocket: probe points on voxel centres and the grid that tabulates them.
 * Eq. 1 takes, for each ligand atom, the minimum squared distance to the
 * pocket's points (Sec. 3.1: the PASS probe-sphere centres). The library
 * tabulates that minimum on the voxel centres in grid units,
 *   K(v) = max(min_j |v - p_j|^2, 1),
 * an exact integer (the floor at one voxel spacing squared keeps Eq. 1's
 * denominator positive).
 *   nx, ny, nz  grid size, 2..DOCK_MAX_GRID each
 *   h           voxel edge (Å), > 0
 *   origin      position of voxel (0,0,0)'s centre (Å)
 *   centre      pocket centre (Å); initial poses put the ligand centroid here
 *   K           optional host array nx*ny*nz (x fastest) used as the field as
 *               is (values >= 1); NULL: the field is built on the GPU from pts
 *   pts         host array 3*npts of voxel indices (x, y, z) inside the grid
 *   npts        >= 1 unless K is given */
typedef struct {
    int nx, ny, nz;
    double h;
    double origin[3];
    double centre[3];
    const uint16_t* K;
    const int32_t* pts;
    int npts;
} dock_pocket;

/* A batch of ligands in CSR form, host arrays (Sec. 2: atoms, covalent bonds
 * and the rotamers among them).
 *   n          number of ligands (>= 0)
 *   atom_off   n+1 offsets; ligand b owns atoms [atom_off[b], atom_off[b+1]),
 *              1..DOCK_MAX_ATOMS of them
 *   xyz        3*atom_off[n] floats, x y z per atom (Å)
 *   bond_off   n+1 offsets into bonds
 *   bonds      2*bond_off[n] ligand-local atom indices (u, v)
 *   rot_off    n+1 offsets into rot
 *   rot        ligand-local bond indices of the rotatable bonds, in sweep
 *              order; each must split its ligand into two fragments
 *   id_base    ligand id of ligand 0 (seeds its initial orientations)
 *   ids        optional n ids (overrides id_base + b) */
typedef struct {
    int n;
    const int32_t* atom_off;
    const float* xyz;
    const int32_t* bond_off;
    const int32_t* bonds;
    const int32_t* rot_off;
    const int32_t* rot;
    int64_t id_base;
    const int64_t* ids;
} dock_ligand_batch;

/* Knobs (Sec. 3.3 and Alg. 2, plus the poses and pose clipping).
 *   hp_step, lp_step   high/low precision angle steps, degrees in [1, 360];
 *                      a sweep tries angles k*step < 360, k >= 1
 *   threshold          fragments with (atoms in fragment / atoms in ligand)
 *                      <= threshold take lp_step, others hp_step
 *   repetitions        passes of the whole greedy procedure, >= 0
 *   n_poses            rigid initial orientations, 1..DOCK_MAX_POSES; pose 0
 *                      is the input conformer, the others are seeded uniform
 *                      random rotations about the centroid (SplitMix64 +
 *                      Shoemake quaternions)
 *   enable_refinement  tile peeling of Alg. 2 / Eq. 2-3 for hp fragments
 *   clip_box           1: a candidate with a moving atom outside the grid is
 *                      infeasible and an initial pose with an atom outside is
 *                      skipped; 0: lookups clamp to the box and add the
 *                      squared distance outside it
 *   bump_thr           Å; a candidate is infeasible when an atom pair whose
 *                      distance depends on the torsion is closer than this
 *   score_mode         0 nearest voxel, 1 trilinear interpolation of K,
 *                      2 exact: Eq. 1's inner minimum over the pocket's
 *                      probe points themselves, O(l p) per candidate (the
 *                      paper's own cost profile; needs the pocket's pts;
 *                      runs with 12 angles per chunk)
 *   refine_steps       ascent steps of dock_refine (0..1000); dock_run ignores it
 *   seed               seed of the initial orientations
 *   plain_mode         1: one launch per (pocket, ligand) pair, no bucketing
 *                      and no graph (the comparison form); 0: batched */
typedef struct {
    double hp_step, lp_step, threshold;
    int repetitions, n_poses;
    int enable_refinement;
    int clip_box;
    double bump_thr;
    int score_mode;
    int refine_steps;
    uint64_t seed;
    int plain_mode;
} dock_knobs;

/* One (pocket, ligand) result.
 *   score   best overlap score o = l / sum_i D_i (Eq. 1, Å^-2) over the
 *           initial poses after the sweep; 0 when status != 0
 *   pose    index of the initial pose that reached it (ties: lowest), -1
 *   status  0 ok, 1 every initial pose was skipped (outside the box) */
typedef struct {
    float score;
    int32_t pose;
    int32_t status;
    int32_t reserved;
} dock_result;

/* Create a context on CUDA device `device`; *out receives it. */
int dock_create(dock_ctx** out, int device);

/* Release every device buffer and the context itself. NULL is ignored. */
void dock_destroy(dock_ctx* ctx);

/* Text of the last error on this context ("" when none). Owned by ctx. */
const char* dock_last_error(const dock_ctx* ctx);

/* Upload a pocket and build its field K on the GPU (Eq. 1, inner minimum),
 * unless p->K is given. *pocket_id receives its handle. Synchronous. The
 * pocket holds, on the device, K (2 bytes per voxel), a padded 32-bit copy
 * for nearest-voxel lookups ((n+32)^3 x 4 bytes) and the 2x2x2 corners of
 * every voxel for the trilinear score (16 bytes per voxel): about 54 MB for
 * a 128^3 grid, 8.2 MB for 64^3. */
int dock_init_pocket(dock_ctx* ctx, const dock_pocket* p, int* pocket_id);

/* Copy a pocket's field back to host memory K (nx*ny*nz uint16, x fastest). */
int dock_pocket_field(dock_ctx* ctx, int pocket_id, uint16_t* K);

/* Upload a ligand batch: checks the topology, finds the two fragments of
 * every rotatable bond (Alg. 1: one on each side of the bond, the left one
 * holding the bond's lower atom index) and copies atoms and fragment
 * tables to the GPU. *batch_id receives its handle. Synchronous.
 * Errors: DOCK_ERR_INVALID_ARG (sizes, indices), DOCK_ERR_TOPOLOGY. */
int dock_upload_ligands(dock_ctx* ctx, const dock_ligand_batch* b, int* batch_id);

/* Free a batch's device memory. */
int dock_release_batch(dock_ctx* ctx, int batch_id);

/* Dock every ligand of the batch into every listed pocket (Alg. 2 per
 * (pocket, ligand, initial pose); best pose per pair).
 *   pocket_ids, npockets   host array of pocket handles (>= 1)
 *   k                      knobs
 *   out                    npockets*n results, pocket-major (caller-owned)
 *   xyz_out                NULL, or npockets*3*atom_off[n] floats: the best
 *                          pose's coordinates (Å) per pair, pocket-major
 *   out_on_device          0: out/xyz_out are host memory and the call waits
 *                          for the results; 1: device memory, written in
 *                          stream order and the call returns at once
 *   stream                 cudaStream_t to run on (NULL: the legacy stream)
 * Device memory for the run is allocated by the library on first use and
 * reused; the batched form replays a CUDA graph per (batch, knobs, pockets). */
int dock_run(dock_ctx* ctx, int batch_id, const int32_t* pocket_ids, int npockets, const dock_knobs* k,
             dock_result* out, float* xyz_out, int out_on_device, void* stream);

/* Dock a ligand database held in host memory: the same results as
 * dock_upload_ligands + dock_run (out_on_device 0) + dock_release_batch on the
 * whole database, computed chunk by chunk with the host preparation and the
 * upload of the next chunk overlapping the device sweep of the current one
 * (two pipeline stages; their device and pinned host buffers stay with the
 * context and are reused by later calls).
 *   b                      the database (same layout and checks as
 *                          dock_upload_ligands; a bad ligand is reported by
 *                          the chunk holding it)
 *   pocket_ids, npockets   host array of pocket handles (>= 1)
 *   k                      knobs (plain_mode is ignored: the chunks always
 *                          run the batched form)
 *   chunk                  ligands per chunk (>= 1; more than n means one)
 *   out                    npockets*n results, pocket-major, host memory
 *   xyz_out                NULL, or npockets*3*atom_off[n] floats (host)
 *   stream                 cudaStream_t of the sweeps (NULL: legacy stream)
 * Waits for every chunk. dock_last_stats then reports the work of the whole
 * database and sweep_ms = -1 (not timed). Errors as dock_upload_ligands and
 * dock_run; results already written for earlier chunks stay in out. */
int dock_run_database(dock_ctx* ctx, const dock_ligand_batch* b, const int32_t* pocket_ids, int npockets,
                      const dock_knobs* k, int chunk, dock_result* out, float* xyz_out, void* stream);

/* Per-candidate trace of one run on one pocket, for parity checks against a
 * reference implementation. Every pointer is device memory (nullable except
 * chosen_k). Sweep index of (ligand b, pose p, sweep s):
 *     sweep_base[b] + p * nsweep[b] + s,  nsweep[b] = repetitions * 2 * T_b,
 *     sweep_base[b] = n_poses * sum_{b' < b} nsweep[b'],
 * sweeps ordered repetition, rotatable bond, then left before right.
 * Candidate slot j of a sweep is at sweep_index * pmax + j; slot 0 is the
 * incumbent (angle 0), slot k >= 1 the angle k*step of a flat sweep; with tile
 * peeling slots 1..360/x are the tile centres and the next x/step slots the
 * angles of the best tile.
 *   chosen_k     committed slot per sweep
 *   cand_S       S = sum_i D_i in grid units per slot (o = l / (h^2 S))
 *   cand_status  1 feasible, 0 bump, -1 outside box, -2 slot not evaluated
 *   pose_S       final S per (ligand, pose) (b * n_poses + p); pose_status
 *                0 ok, 1 skipped; pose_init_S initial S
 *   init_xyz, pose_xyz  per (ligand, pose) coordinates (Å) at
 *                (atom_off[b] * n_poses + p * l_b) * 3 */
typedef struct {
    int32_t pmax;
    const int64_t* sweep_base;
    int32_t* chosen_k;
    float* cand_S;
    int32_t* cand_status;
    float* pose_S;
    float* pose_init_S;
    int32_t* pose_status;
    float* init_xyz;
    float* pose_xyz;
} dock_trace;

/* dock_run on one pocket with the trace above recorded (same kernels, trace
 * stores switched on). Synchronous. */
int dock_run_trace(dock_ctx* ctx, int batch_id, int pocket_id, const dock_knobs* k, const dock_trace* tr,
                   dock_result* out, void* stream);

/* Candidate slots per sweep of the trace layout for these knobs. */
int dock_trace_pmax(const dock_knobs* k);

/* Tile shape of the sweep kernel. lanes_per_pose (1, 2, 4, 8) lanes share a
 * pose and split its moving atoms (a ligand whose poses would not fit the
 * warp's coordinate slice gets more, and so, with the nearest-voxel score
 * and lanes_per_pose not forced, does a ligand whose pose group would
 * outlast the average load of the launch's warps); angles_per_chunk (8, 12,
 * 18, 36) angles a lane
 * keeps in registers; warps_per_cta. dock_set_tile forces a shape for the
 * batched form (0 fields keep the current choice); dock_autotune times the
 * shapes on a sample of the batch and keeps the fastest for (batch, knobs). */
typedef struct {
    int lanes_per_pose;
    int angles_per_chunk;
    int warps_per_cta;
} dock_tile;

int dock_set_tile(dock_ctx* ctx, const dock_tile* t);
int dock_get_tile(const dock_ctx* ctx, dock_tile* t);
int dock_autotune(dock_ctx* ctx, int batch_id, int pocket_id, const dock_knobs* k, dock_tile* best, void* stream);

/* Work and timing of the last dock_run, counted from the topology and knobs:
 *   candidates       candidate angles evaluated, over all (pocket, ligand,
 *                    pose, sweep), excluding the incumbents
 *   atom_updates     (candidate, moving atom) pairs placed and looked up in
 *                    the field: each is one rotation and one field lookup;
 *                    excludes lookups_skipped
 *   pair_bounds      (sweep, moving atom, partner atom) circle bound tests of
 *                    the bump check
 *   bump_pairs       (candidate, atom pair) distance tests a bump check
 *                    without the circle bound would make
 *   kernel_launches  CUDA kernels launched by the call
 *   sweep_ms         device time of the sweep kernel(s) of the call, from
 *                    CUDA events recorded around them on the call's stream
 *                    (waits for the call to finish)
 *   pose_reps_skipped  (pose, repetition) pairs not computed: a repetition
 *                    that commits no angle for a pose leaves it where it
 *                    was, so each further repetition would repeat it
 *                    exactly; a pose that starts outside the box (clip_box)
 *                    computes none; the counts above exclude that work
 *   lookups_skipped  (candidate, moving atom) lookups not made because the
 *                    bump check had already rejected every candidate of
 *                    their block of angles for every pose computed in the
 *                    warp (nearest-voxel and trilinear scores) */
typedef struct {
    uint64_t candidates;
    uint64_t atom_updates;
    uint64_t pair_bounds;
    uint64_t bump_pairs;
    uint64_t kernel_launches;
    double sweep_ms;
    uint64_t pose_reps_skipped;
    uint64_t lookups_skipped;
} dock_stats;

int dock_last_stats(const dock_ctx* ctx, dock_stats* s);

/* Rates that bound the sweep, measured on the context's device (for the
 * roofline of the measurement; not part of docking):
 *   fma_per_s           FP32 fused multiply-adds per second (scalar fmaf,
 *                       eight independent chains per thread, 2,048 threads
 *                       per SM)
 *   ffma2_per_s         the same with packed two-wide FP32 multiply-adds,
 *                       counting both
 *   tex_field_per_s     point-sampled fetches per second from the pocket's
 *                       padded-field texture, coordinates spread over the
 *                       whole field (L2-resident)
 *   tex_local_per_s     the same within a 16^3-voxel cube per warp
 *                       (L1-resident: the locality of one ligand's poses)
 *   l2_sectors_per_s    random 32-byte sector loads per second from a 64 MiB
 *                       buffer held in L2
 * Each is timed with CUDA events on `stream` after a warm-up launch; the call
 * allocates 65 MiB of device memory for its duration and waits. */
typedef struct {
    double fma_per_s;
    double ffma2_per_s;
    double tex_field_per_s;
    double tex_local_per_s;
    double l2_sectors_per_s;
} dock_peaks;

int dock_measure_peaks(dock_ctx* ctx, int pocket_id, dock_peaks* out, void* stream);

/* dock_run for callers that cannot allocate device memory.
 *
 * The paper has no counterpart: this exists for the library's users. Some
 * callers must not call cudaMalloc or cudaFree on the docking path: a
 * serving loop whose device memory is carved up in advance by its own pool
 * or arena and is capped there, or a caller that cannot afford the device
 * synchronisation an allocation or a free may bring. dock_run may allocate
 * its scratch on first use or when a batch grows; this call never does. Its
 * scratch (work-queue head, angle tables, task list, per-pose keys and
 * coordinates) lives in one file-scope device array of about 50 MiB, which
 * every GPU that loads the library holds until the process exits.
 *
 * Same docking as dock_run on ONE pocket, with results equal to dock_run's
 * bit for bit in every score mode when both run the same tile shape (the
 * default, or the one dock_set_tile forces; a shape found by dock_autotune is
 * not used here). The batch and pocket must already be uploaded
 * (dock_upload_ligands and dock_init_pocket do allocate; do them at set-up).
 * The call enqueues its kernels on `stream` and returns without waiting:
 * outputs are device memory written in stream order, and no host memory is
 * read once the call has returned (the angle tables travel as kernel
 * parameters; the step choice of Alg. 2 is made on the device).
 *   out      device array of n dock_result (n = ligands in the batch)
 *   xyz_out  NULL or device array of 3*atom_off[n] floats (best pose, Å)
 * Limits per call: n_poses * n <= 131072 and n_poses * atom_off[n] <=
 * 4194304, and at most 361 angles per sweep; larger runs fail with
 * DOCK_ERR_INVALID_ARG before anything is launched.
 * Cost: the work list runs in ligand order rather than longest first, and
 * every ligand gets as many pose groups as the batch's largest ligand needs
 * (the extra ones idle), so on batches of mixed sizes it is slower than
 * dock_run.
 * The first call on a device looks up the array's device address there (once
 * per device, with that device current); make that first call before any
 * stream capture. The address stays valid for the life of the device's
 * context: after cudaDeviceReset, do not call this entry point again in the
 * same process. Every call shares the one array and leaves its contents
 * behind: the call clears what must start at zero itself, and calls whose
 * work overlaps on the GPU (other streams, other threads) race on it; keep
 * them ordered. dock_last_stats is not updated by this call. */
int dock_run_static(dock_ctx* ctx, int batch_id, int pocket_id, const dock_knobs* k, dock_result* out,
                    float* xyz_out, void* stream);

/* ------------------------------------------------------------------------
 * Local refinement and the differentiable score (not in the paper, which
 * only mentions steepest descent; built on the trilinear form of Eq. 1).
 *
 * Score: S = sum_i D(x_i), D the trilinear interpolant of K between voxel
 * centres (grid units); outside the box D is taken at the clamped position,
 * plus the squared excess in grid units when clipping is off;
 * o = l / (h^2 S) (Å^-2).
 *
 * Pose degrees of freedom of ligand b: q = (t, omega, theta_1..theta_T),
 * T = its rotatable bonds in the batch's order. theta_k turns the side of
 * bond k away from atom 0 about the axis from the bond's other atom to its
 * own bond atom (right-handed), deepest bond first; then the pose rotates by
 * the rotation vector omega (radians) about the centroid g of the input
 * coordinates x and moves by t (Å):  z = g + R(omega) (tau(x) - g) + t.
 *
 * Every pointer below is device memory; calls are asynchronous on `stream`
 * unless stated otherwise. Coordinates use the batch's atom_off layout
 * (3 floats per atom, Å), per pocket where a call takes several pockets
 * (pocket-major, as dock_run's xyz_out).
 * ------------------------------------------------------------------------ */

/* Ligand count, atom count, largest ligand and largest torsion count of a
 * batch (host pointers; any may be NULL). q arrays use a stride of at least
 * 6 + tmax floats per ligand. */
int dock_batch_info(dock_ctx* ctx, int batch_id, int* n, int* natoms, int* lmax, int* tmax);

/* o per ligand (n floats) of the poses xyz on one pocket. clip: 1 the
 * box-clamped interpolant, 0 plus the outside penalty. */
int dock_score_trilinear(dock_ctx* ctx, int batch_id, int pocket_id, int clip, const float* xyz, float* o,
                         void* stream);

/* Adjoint of dock_score_trilinear: grad_xyz (3 * natoms floats) =
 * grad_o[b] * d o_b / d x_i, with grad_o NULL meaning ones. */
int dock_score_trilinear_grad(dock_ctx* ctx, int batch_id, int pocket_id, int clip, const float* xyz,
                              const float* grad_o, float* grad_xyz, void* stream);

/* z = the pose x moved by q (n * qstride floats, qstride >= 6 + tmax). */
int dock_dof_apply(dock_ctx* ctx, int batch_id, const float* x, const float* q, int qstride, float* z, void* stream);

/* Adjoint of dock_dof_apply at (x, q): grad_q = J(q)^T grad_z, where
 *   d/dt = sum_i g_i,  d/domega = Jl(omega)^T sum_i (z_i - g - t) x g_i
 *   (Jl the left Jacobian of the exponential map), d/dtheta_k = axis_k .
 *   sum over the moving side of (z_i - z_c) x g_i with the axis taken in z.
 * Slots of grad_q past 6 + T_b are set to 0. */
int dock_dof_grad(dock_ctx* ctx, int batch_id, const float* x, const float* q, int qstride, const float* grad_z,
                  float* grad_q, void* stream);

/* Local refinement of one pose per (pocket, ligand): k->refine_steps steps
 * of gradient ascent on the trilinear o from the poses xyz_in (e.g. dock_run's
 * xyz_out). A step moves along d o / d q, scaled so that the largest
 * first-order atom displacement is lambda Å; it is kept only if S drops, no
 * pair moved by a torsion (Alg. 1's bump pairs, all rotatable bonds) comes
 * closer than k->bump_thr, and (k->clip_box) every atom stays inside the
 * box. lambda starts at 0.25 Å, grows by 1.5 after a kept step (at most
 * 1 Å) and halves after a rejected one. Pairs whose start pose lies outside
 * the box with clipping on are returned unchanged with status 1.
 *   xyz_in, xyz_out   npockets * 3 * atom_off[n] floats (may alias: no)
 *   out               npockets * n results: score = refined o, pose = -1,
 *                     status 0 refined / 1 skipped
 *   on_device         1: every pointer is device memory, the call returns
 *                     at once; 0: host memory, the call waits
 * Uses k->refine_steps, k->clip_box and k->bump_thr; the trilinear score
 * regardless of k->score_mode. */
int dock_refine(dock_ctx* ctx, int batch_id, const int32_t* pocket_ids, int npockets, const dock_knobs* k,
                const float* xyz_in, dock_result* out, float* xyz_out, int on_device, void* stream);

/* Per-step record of dock_refine on one pocket, host arrays, for parity
 * checks. Index of (ligand b, step s): b * steps + s.
 *   gstride   stride of G (>= 6 + tmax)
 *   G         d o / d q at the step's start pose (n * steps * gstride)
 *   D         largest first-order atom displacement per unit of G (Å)
 *   lam       step length used (Å)
 *   S_new     S of the trial pose (grid units)
 *   verdict   bit0 S_new < S, bit1 bump-free, bit2 inside the box
 *   accept    1 when the trial pose was kept
 *   S_start, S_final, status   per ligand */
typedef struct {
    int32_t gstride;
    float* G;
    float* D;
    float* lam;
    float* S_new;
    int32_t* verdict;
    int32_t* accept;
    float* S_start;
    float* S_final;
    int32_t* status;
} dock_refine_trace_buf;

/* dock_refine on one pocket with the record above. Host arrays, synchronous. */
int dock_refine_trace(dock_ctx* ctx, int batch_id, int pocket_id, const dock_knobs* k, const float* xyz_in,
                      const dock_refine_trace_buf* tr, dock_result* out, float* xyz_out);

#ifdef __cplusplus
}
#endif

#endif /* GEODOCK_H */
