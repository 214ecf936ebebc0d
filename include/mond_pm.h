/*
 * mond_pm.h -- C ABI of the GB300 (sm_103a) MOND particle-mesh force pipeline.
 *
 * Method: Visser, Eijt & de Nijs, "Fast particle-mesh code for Milgromian
 * dynamics" (A&A 2023, arXiv:2312.02968). One time step is
 *   deposit (Eq. smooth) -> field solve (Sect. 2.1 iteration, App. Flow steps
 *   3-9) -> gather (Eq. gi) -> leapfrog kick and drift (Eq. motion).
 *
 * Conventions shared by every call:
 *  - Mesh: the FFT domain is n_f^3 pixels of width s = box / n, with
 *    n_f = n (pad = 1) or n_f = 2n (pad = 2: the physical n^3 sits in the
 *    centre of a zero-padded periodic domain). The whole iteration is periodic
 *    on n_f^3 (Sect. 3: periodic lattice with empty margin).
 *  - Scalar mesh fields are float32 [z][y][x] (x fastest), n_f^3 values;
 *    vector fields are three such planes, component x first.
 *  - Particles are borrowed device arrays in [N][3] layout: int32 cell (the
 *    FFT-domain pixel of the nearest pixel centre, 0..n_f-1 on each axis),
 *    float32 offset from that centre in pixels, in [-1/2, 1/2], float32
 *    velocity (length per time), and float32 mass [N]. Physical position is
 *    (cell - n_f/2 + offset) * s.
 *  - Every call enqueues work on the handle's CUDA stream and returns without
 *    synchronising, unless its comment says it synchronises.
 *  - Every call returns MOND_OK (0) or a negative error code. Errors found on
 *    the device (a particle outside the domain, a non-finite field) are
 *    latched in a device status word and returned by the next call that
 *    synchronises (mond_pm_sync, mond_pm_diagnostics, mond_pm_get_field).
 *    mond_pm_last_error() describes the most recent error.
 *
 * Ownership: the caller allocates all device memory. The handle only carves
 * the caller's workspace (mond_pm_workspace_bytes) and borrows the particle
 * arrays; it frees neither. The library calls no cudaMalloc.
 */
#ifndef MOND_PM_H
#define MOND_PM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mond_pm* mond_pm_t;

typedef struct {
  int32_t n;   /* physical mesh side; n_f = n * pad must be 2^a 3^b, 16 <= n_f <= 512 */
  int32_t pad; /* 1 or 2 */
} mond_pm_grid;

/* Interpolation function mu (Eq. mu and Sect. 4): deep mu(x) = x; simple
 * mu(x) = x/(1+x); standard mu(x) = x/sqrt(1+x^2); Newton mu = 1. */
enum { MOND_MU_DEEP = 0, MOND_MU_SIMPLE = 1, MOND_MU_STANDARD = 2, MOND_MU_NEWTON = 3 };

/* Initial H of the iteration: zero (App. Flow step 7), the H of the previous
 * solve (Sect. 5.2 item iv), a caller-supplied guess projected onto its
 * divergence-free part, or a caller-supplied guess used as given.
 * MOND_WARM_INCREMENT is the incremental solve of Sect. 5.2 item v: the
 * fields' increments for the change of the deposit since the base state, with
 * the nu and mu steps linearised about that state (see
 * mond_pm_set_increment_workspace). */
enum { MOND_WARM_NONE = 0, MOND_WARM_PREV = 1, MOND_WARM_GUESS = 2, MOND_WARM_GUESS_RAW = 3,
       MOND_WARM_INCREMENT = 4 };

/* Mesh fields readable with mond_pm_get_field. */
enum {
  MOND_FIELD_RHO = 0,    /* density from the last deposit, 1 plane */
  MOND_FIELD_GN = 1,     /* Newtonian field g_N of the last solve, 3 planes */
  MOND_FIELD_H = 2,      /* H state: the last H formed by a solve (warm-start state), 3 planes */
  MOND_FIELD_PHI = 3,    /* MOND potential phi of the last solve, 1 plane (needs MOND_OPT_KEEP_PHI) */
  MOND_FIELD_ACC = 4,    /* acceleration mesh a = -grad_FD phi of the last solve, 3 planes (node-smoothed
                            when the solve ran with MOND_OPT_GATHER 1 or 3) */
  MOND_FIELD_SMOOTH = 5, /* node-smoothed acceleration of the last mond_pm_smooth, 3 planes */
  MOND_FIELD_GM = 6      /* base g_M of an incremental solve: the curl-free g_M of the last iteration of the
                            last solve, 3 planes (needs the increment workspace; MOND_ESTATE otherwise) */
};

/* Error codes. */
enum {
  MOND_OK = 0,
  MOND_EINVAL = -1,    /* bad argument (size, kind, width, pointer, alignment) */
  MOND_ENOMEM = -2,    /* workspace too small */
  MOND_ECUDA = -3,     /* a CUDA runtime call failed */
  MOND_EOVERFLOW = -4, /* fixed-point bound violated (cannot happen for N < 2^31) */
  MOND_EDOMAIN = -5,   /* a particle's cell or offset is outside the domain; it was skipped */
  MOND_ENAN = -6,      /* a non-finite value appeared in a field or a particle */
  MOND_ETIMEOUT = -7,  /* a bounded device wait gave up (kernel returned early) */
  MOND_ESTATE = -8     /* call out of order (no particles bound, no solve yet, ...) */
};

/* Options for mond_pm_set_option. */
enum {
  MOND_OPT_KEEP_PHI = 1,  /* value 1: also form the potential phi in the final pass */
  MOND_OPT_TRACK_DH = 2,  /* value 1: record ||H_j - H_{j-1}|| / ||g_N|| per iteration (costs one reduction) */
  MOND_OPT_USE_GRAPH = 3, /* value 1: mond_pm_step runs as a CUDA graph, captured on first use and again
                             when an argument, option or binding changes; needs a non-default stream and
                             is bypassed while MOND_OPT_TIMING is on (default 0) */
  MOND_OPT_TIMING = 4,    /* value 1: bracket every launch with CUDA events (see mond_pm_kernel_stats) */
  MOND_OPT_PIPELINED = 5, /* value 1 (default): y/z passes stream tiles with TMA through a two-stage ring;
                             0: one tile per CTA with plain loads (same results) */
  MOND_OPT_CHUNK = 6,     /* particles per deposit/gather work item: a power of two in 256..4096
                             (default 1024; same results) */
  MOND_OPT_GATHER = 7,    /* force at the particles. 0 (default): Eq. gi, the ball sum at each particle.
                             1 or 3: the mesh-interpolating gather -- the final pass of a solve (n_iter >= 1)
                             also multiplies the acceleration spectrum by the smoothing spectrum, so that
                             MOND_FIELD_ACC holds the node-smoothed field of mond_pm_smooth, and the force
                             at a particle is the linear (1) or Keys cubic (3, a = -1/2) interpolation of
                             that field at its position: an approximation of Eq. gi whose error the caller
                             measures against variant 0. A gather whose variant disagrees with the mesh
                             the last solve made fails with MOND_ESTATE. */
  MOND_OPT_TEST_LOST_LOAD = 8, /* tests of the bounded device waits only. value t + 1 (t >= 0): in the next
                             pipelined y-pass the tile copy of tile t is never issued, so the wait for it
                             gives up after a short bound, the CTA waits for the copy it did issue and
                             stops, and the next synchronising call returns MOND_ETIMEOUT (the fields of
                             that solve are invalid; the handle stays usable). One-shot: cleared by that
                             launch. 0: off. Needs MOND_OPT_PIPELINED 1 and no graph replay. */
  MOND_OPT_CYCLE_MEAN = 9,    /* value 1: a solve with n_iter >= 2 (plain or warm-started, not incremental)
                             takes as its potential the mean of the potentials of its last two iterations'
                             curl-free steps, phi^ = (phi^_{K-1} + phi^_K)/2. Near zeros of the field the
                             iteration of Sect. 2.1 ends in a period-2 cycle (its iterates alternate about
                             the solution of the discretised equation); the mean is the cycle's midpoint.
                             Not in the paper. Costs one half-spectrum plane written and read. Needs
                             MOND_OPT_PIPELINED 1 (default 0) */
  MOND_OPT_FOLD = 10,         /* value 1 (default): where the pipelined passes run and the side allows it
                             (every supported side but 16 and 48), the curl-free, final and Newton steps
                             carry one scalar and its z-derivative between their y- and z-passes instead
                             of three components (the gradient form of their operators, with the axes on a
                             Nyquist plane kept apart); 0: three components throughout. Same results up to
                             FP32 rounding order. */
  MOND_OPT_GRID_CAP = 11      /* value c > 0: the persistent kernels of a step (pipelined y/z passes,
                             deposit, gather) launch at most c CTAs, leaving the rest of the GPU to
                             kernels that run beside them (independent systems on their own streams,
                             a batch); 0 (default): as many as fit the GPU. Same results. */
};

/* Per kernel class: launches, device time between the events around each
 * launch, and the algorithmic bytes the launches must move (each input
 * element read once, each output element written once). */
typedef struct {
  char name[32];
  int64_t launches;
  double ms;
  double bytes;
} mond_pm_kstat;

typedef struct {
  double mass;          /* sum of m_i */
  double momentum[3];   /* sum m_i v_i */
  double com[3];        /* centre of mass (physical coordinates) */
  double ang_mom[3];    /* sum m_i (x_i - com) x v_i */
  double e_kin;         /* sum m_i |v_i|^2 / 2 */
  double e_pot;         /* s^3 sum rho phi (needs MOND_OPT_KEEP_PHI and a solve), else NaN */
  double rho_mass;      /* s^3 sum rho of the last deposit */
  int32_t n_iter_done;  /* iterations run by the last solve */
  int32_t pad_;
  double dH[64];        /* ||H_j - H_{j-1}|| / ||g_N|| per iteration (MOND_OPT_TRACK_DH), NaN otherwise */
} mond_pm_diag;

/* Bytes of device workspace a handle with this grid and kernel width needs
 * for up to max_particles particles. Returns MOND_EINVAL for an unsupported
 * grid or width. */
int mond_pm_workspace_bytes(mond_pm_grid grid, double kernel_width, int64_t max_particles, size_t* bytes);

/* Create a handle. box: physical side of the n^3 mesh (s = box/n); a0:
 * Milgrom's constant; G: Newton's constant; mu_kind: MOND_MU_*;
 * kernel_width: sigma of the Gaussian of Eq. smooth in pixels (0.75..2; the
 * paper uses 1; the ball of taps is |d| < 4 sigma, Sect. 3.1); cuda_stream: a
 * cudaStream_t (NULL = default stream); workspace: device memory of at least
 * mond_pm_workspace_bytes (256-byte aligned), owned by the caller and kept
 * alive until mond_pm_destroy. Builds the lookup table of Sect. 3.1 on the
 * host and uploads it (synchronises once). */
int mond_pm_create(mond_pm_grid grid, double box, double a0, double G, int mu_kind, double kernel_width,
                   void* cuda_stream, void* workspace, size_t workspace_bytes, int64_t max_particles,
                   mond_pm_t* out);

/* Release the handle (not the workspace, not the particles). Synchronises. */
int mond_pm_destroy(mond_pm_t h);

/* Set an option (MOND_OPT_*). */
int mond_pm_set_option(mond_pm_t h, int option, int64_t value);

/* Borrow particle arrays (device pointers, layout above), N <= max_particles.
 * Scans the masses for the fixed-point scale (synchronises once). The arrays
 * cell, offset and vel are updated in place by gather_push / half_kick. */
int mond_pm_bind_particles(mond_pm_t h, int64_t N, int32_t* cell, float* offset, float* vel, const float* mass);

/* Mass deposit, Eq. smooth restricted to the ball around each particle's
 * cell (Sect. 3.1; App. Flow main loop steps 1-2) in a fixed-point rule that
 * makes the result independent of order and bit-identical to the CPU oracle:
 * per-axis weights round(2^24 g1) from a table indexed by the offset rounded
 * to 2^-16 px, combined in integers, accumulated in int64 units of
 * 2^-Kacc mass; rho = float(double(acc) * 2^-Kacc / s^3). Also bins the
 * particles by 8^3 mesh tile for the gather. */
int mond_pm_deposit(mond_pm_t h);

/* Use a mesh density instead of a deposit for the next solves: rho (device
 * float32, n_f^3, mass per s^3) is copied in; the next mond_pm_deposit
 * replaces it. Particle calls (gather, push) need a deposit. */
int mond_pm_set_density(mond_pm_t h, const float* rho);

/* Field solve (Sect. 2.1 iteration; App. Flow steps 3-9) on the last
 * deposit: Newtonian field, then n_iter iterations of
 * F = g_N + H, g_M = nu(|F|/a0) F, curl-free projection, F = mu(|g_M|/a0) g_M,
 * H = F - g_N, divergence-free projection; the last iteration stops after the
 * curl-free projection and the acceleration mesh a = -grad_FD phi is formed.
 * n_iter = 0 gives the Newtonian solve (a = g_N). warm: MOND_WARM_NONE
 * (H = 0), MOND_WARM_PREV (H of the previous solve), MOND_WARM_GUESS
 * (H_guess: device float32, 3 planes; it is projected onto its
 * divergence-free part first) or MOND_WARM_GUESS_RAW (H_guess used as
 * given, once: the H state is left as it was). With MOND_WARM_PREV or
 * MOND_WARM_GUESS the last iteration also completes the H update so the next
 * solve can start from it. The Newtonian field is computed once
 * per density: a solve on the density of the previous solve (no deposit or
 * mond_pm_set_density in between) starts from the stored g_N.
 * MOND_WARM_INCREMENT (n_iter >= 1) runs the incremental solve (Sect. 5.2
 * item v) on the deposit's change since the base: the density increment is the
 * difference of the two int64 accumulators (exact), converted by the density
 * rule; dg_N is its Newtonian field; then n_iter iterations of
 * dF = dg_N + dH, dg_M = curl-free part of Jnu(F0) dF,
 * dH = divergence-free part of Jmu(g_M0) dg_M - dg_N, with
 * J f(P) d = f(p) d + p f'(p) (u.d) u (p = |P|/a0, u = P/|P|; the identity for
 * the Newtonian kind, 0 where P = 0), F0 = g_N + H and g_M0 of the base. The
 * last iteration adds the increments of the acceleration mesh (and phi), g_N,
 * g_M and H to the base, which becomes this solve's state.
 * MOND_ESTATE when no base is valid (see mond_pm_set_increment_workspace).
 * 0 <= n_iter <= 64. */
int mond_pm_solve_field(mond_pm_t h, int n_iter, int warm, const float* H_guess);

/* Workspace of the incremental solve (Sect. 5.2 item v): the base deposit
 * (int64, n_f^3), the base g_M and the increment's g_N (float32, 3 planes
 * each). mond_pm_increment_workspace_bytes gives its size for a grid
 * (MOND_EINVAL for a bad grid). mond_pm_set_increment_workspace attaches ws
 * (device memory, 256-byte aligned, caller-owned, unused by the handle once
 * detached; NULL detaches); errors: MOND_EINVAL (misaligned), MOND_ENOMEM
 * (too small). While one is attached, every solve with n_iter >= 1 (other than
 * MOND_WARM_GUESS_RAW, and not on a density set with mond_pm_set_density) also
 * completes the H update, stores the curl-free g_M of its last iteration and
 * copies the deposit: the base of the next MOND_WARM_INCREMENT solve. The base
 * is dropped by mond_pm_set_density, mond_pm_set_h_state,
 * mond_pm_set_dipole_layer, a Newtonian or MOND_WARM_GUESS_RAW solve, and
 * attaching; an incremental solve needs the Kacc, MOND_OPT_GATHER and
 * MOND_OPT_KEEP_PHI of its base. */
int mond_pm_increment_workspace_bytes(mond_pm_grid grid, size_t* bytes);
int mond_pm_set_increment_workspace(mond_pm_t h, void* ws, size_t bytes);

/* Node-smoothed acceleration: the periodic discrete convolution of the
 * acceleration mesh with the ball-truncated Gaussian of Eq. gi, i.e. the force
 * Eq. gi gives a particle sitting exactly on each pixel centre. Written to
 * accel_mesh_out (device float32, 3 planes) when non-NULL and kept for
 * mond_pm_get_field(MOND_FIELD_SMOOTH). */
int mond_pm_smooth(mond_pm_t h, float* accel_mesh_out);

/* Densities from a field of the last solve (Eq. apparentdensity, Sect. 2.1):
 * rho = -(div g) / (4 pi G), the divergence taken with the periodic central
 * difference (f[i+1] - f[i-1]) / (2 s) of the solver's gradients. */
enum {
  MOND_DENS_BARYONIC = 0, /* from g_N: rho_B (the deposit's density seen through the discrete operators) */
  MOND_DENS_APPARENT = 1, /* from the MOND acceleration mesh: rho_A, baryonic plus apparent dark matter */
  MOND_DENS_PHANTOM = 2   /* rho_A - rho_B, the phantom dark matter density */
};

/* Write the density `which` (MOND_DENS_*) of the fields of the last solve to
 * out (device float32, n_f^3 in z, y, x order, 16-byte aligned, caller-owned).
 * Enqueued on the handle's stream; does not synchronise. Errors: MOND_EINVAL
 * (unknown kind, null or misaligned out), MOND_ESTATE (no solve yet). */
int mond_pm_density(mond_pm_t h, int which, float* out);

/* Mass of the density `which` in spherical shells about center (physical
 * (x, y, z); cell i sits at (i - n_f/2) s): out[k] (host, nbins doubles) is the
 * FP64 sum of rho s^3 over the cells whose centre lies at a minimum-image
 * distance r with floor(r / dr) = k, 1 <= nbins <= 4096, dr > 0. The shell of
 * a cell is decided in IEEE double with every operation rounded on its own.
 * The cumulative sum is the enclosed mass M(r) of Eq. totalmass.
 * Synchronises and returns any latched device error. */
int mond_pm_shell_mass(mond_pm_t h, int which, const double center[3], double dr, int nbins, double* out);

/* Eq. totalmass for the box W of cells lo..hi (inclusive per axis, (x, y, z),
 * periodic, 1 <= hi - lo + 1 <= n_f): *out (host) = -(1/(4 pi G)) times the
 * outward flux of the field through the faces of W, the field on a face the
 * mean of the two cells it separates (so that it equals the box sum of
 * mond_pm_density times s^3). Synchronises. */
int mond_pm_box_mass(mond_pm_t h, int which, const int32_t lo[3], const int32_t hi[3], double* out);

/* Replace the H state (MOND_FIELD_H, what MOND_WARM_PREV starts from) by H
 * (device float32, 3 compact planes of n_f^3, read before the call's work
 * completes on the handle's stream; caller-owned). With the particle arrays
 * this is all a run needs to resume: the deposit is exact and the rest of a
 * step is deterministic, so a resumed run continues bit for bit. Enqueued;
 * does not synchronise. Errors: MOND_EINVAL (null H). */
int mond_pm_set_h_state(mond_pm_t h, const float* H);

/* External field by a dipole layer (Sect. 5.3): every later solve adds the
 * density +mass/(n_f^2 s^3) on the last plane of the domain along `axis`
 * (0, 1, 2 for x, y, z) and -mass/(n_f^2 s^3) on the first plane, the planes
 * farthest from a system centred in the domain; the layer's net mass is zero.
 * In Newtonian gravity it makes the field 4 pi G mass s / L^3 along +axis
 * everywhere away from it (L = n_f s); the MOND field follows from the solve.
 * The deposit's density (MOND_FIELD_RHO, the diagnostics) does not include it;
 * g_N and the densities of mond_pm_density do. axis = -1 removes the layer.
 * Enqueues nothing. Errors: MOND_EINVAL (axis outside -1..2, non-finite mass). */
int mond_pm_set_dipole_layer(mond_pm_t h, int axis, double mass);

/* Force at the particles from the acceleration mesh of the last solve
 * (Eq. gi, same ball and Gaussian as the deposit, FP32 weights), then the
 * leapfrog step of Eq. motion: v += g dt; r += v dt; the cell becomes the
 * nearest pixel centre and wraps periodically. Uses the binning of the last
 * deposit, so the particles must not have moved since. */
int mond_pm_gather_push(mond_pm_t h, double dt);

/* As gather_push but velocity only (v += g dt): the initial or final half
 * step of Sect. 3. */
int mond_pm_half_kick(mond_pm_t h, double dt);

/* Force at the particles only (Eq. gi) into g_out (device float32 [N][3]). */
int mond_pm_gather(mond_pm_t h, float* g_out);

/* One time step: deposit, solve_field(n_iter, warm, NULL), gather_push(dt).
 * warm: MOND_WARM_NONE, MOND_WARM_PREV or MOND_WARM_INCREMENT. */
int mond_pm_step(mond_pm_t h, double dt, int n_iter, int warm);

/* ---- batches of independent systems -------------------------------------
 * A batch steps many handles (grids of any supported size, each with its own
 * particles) as one CUDA graph: a fork from the batch stream to every
 * handle's stream, one mond_pm_step of each system on its own stream, and a
 * join back. The graph is captured on the first call and again whenever a
 * step argument, an option or a particle binding of any member changes.
 * The launches of each member are captured from a stream the batch owns for
 * it, so the members are independent branches of the graph whatever streams
 * the handles use; replays run on the batch stream, so a caller that also
 * drives a member directly on its own stream synchronises in between.
 * Ownership: the handles stay owned by the caller and must outlive the batch. */
typedef struct mond_pm_batch* mond_pm_batch_t;

/* Create a batch of n distinct handles; stream: the batch's non-default
 * stream. Errors: MOND_EINVAL (a default stream, a null or repeated handle),
 * MOND_ECUDA; the text is in mond_pm_last_error(NULL). */
int mond_pm_batch_create(int n, const mond_pm_t* handles, void* stream, mond_pm_batch_t* out);

/* Enqueue n_steps graph launches of one step (deposit, solve_field(n_iter,
 * warm NONE, PREV or INCREMENT), gather_push(dt)) of every member on the batch stream.
 * Does not synchronise. */
int mond_pm_batch_step(mond_pm_batch_t b, double dt, int n_steps, int n_iter, int warm);

/* Wait for the batch stream and return the first latched device error of the
 * members. */
int mond_pm_batch_sync(mond_pm_batch_t b);

/* Kernel launches replayed by the batch's graph launches so far. */
int64_t mond_pm_batch_kernel_launches(mond_pm_batch_t b);

/* Synchronise and release the batch (not its handles). */
int mond_pm_batch_destroy(mond_pm_batch_t b);

/* Autotuner: time `trials` steps of length zero (which leave the particles
 * exactly as they are; the H state is reset) for each work-item size in
 * {512, 1024, 2048, 4096} and each pass variant (MOND_OPT_PIPELINED 0/1) on
 * the handle's stream, keep the fastest and report it (either out pointer may
 * be NULL). Synchronises. */
int mond_pm_autotune(mond_pm_t h, int n_iter, int trials, int64_t* chosen_chunk, int* chosen_pipelined);

/* One time step through host memory: copies cell/offset/vel of the N bound
 * particles from the host arrays (pinned memory recommended) to the bound
 * device arrays, runs mond_pm_step, copies cell/offset/vel back and
 * synchronises. The velocities go in on a copy stream of the handle while the
 * deposit and the solve run (the gather waits for them); the other copies are
 * on the handle's stream. Masses are not copied: they are constant and were
 * scanned at bind time. Returns any latched device error. */
int mond_pm_step_host(mond_pm_t h, double dt, int n_iter, int warm, int32_t* cell_host, float* offset_host,
                      float* vel_host);

/* Diagnostics in FP64 (the monitored quantities of Sects. 4.1 and 4.3) into a
 * host struct. Synchronises and returns any latched device error. */
int mond_pm_diagnostics(mond_pm_t h, mond_pm_diag* out);

/* Copy a mesh field (MOND_FIELD_*) into dst (device float32, compact n_f^3
 * per plane). Synchronises and returns any latched device error. */
int mond_pm_get_field(mond_pm_t h, int which, float* dst);

/* Device address of the handle's own buffer of MOND_FIELD_GN, MOND_FIELD_H or
 * MOND_FIELD_ACC (3 compact planes, float32, owned by the handle), for
 * kernels that read a field on the handle's stream without a copy: the
 * contents are those of the last call that wrote the field, in stream order.
 * Does not synchronise. Other fields: MOND_EINVAL. */
int mond_pm_field_ptr(mond_pm_t h, int which, const float** out);

/* Copy the raw int64 deposit accumulator of the last deposit (n_f^3 words)
 * into dst (device) and report Kacc (units are 2^-Kacc mass). Synchronises. */
int mond_pm_get_deposit_acc(mond_pm_t h, uint64_t* dst, int32_t* kacc);

/* Synchronise the stream and return (and clear) any latched device error. */
int mond_pm_sync(mond_pm_t h);

/* Text of the last error on this handle (or of the last failed create when
 * h is NULL). Valid until the next call on the handle. */
const char* mond_pm_last_error(mond_pm_t h);

/* Number of kernels this handle has launched since creation (each graph
 * replay counts its kernels). */
int64_t mond_pm_kernel_launches(mond_pm_t h);

/* Kernel statistics gathered while MOND_OPT_TIMING is on: fills up to cap
 * entries (one per kernel class that ran), sets *count, and resets the
 * statistics. Synchronises. */
int mond_pm_kernel_stats(mond_pm_t h, mond_pm_kstat* out, int cap, int* count);

/* A measurement of the device, not a step of the method: the throughput of
 * no-return shared-memory atomic adds of `bits` = 32 or 64 bits, each thread
 * of a full grid (every SM at its occupancy) adding to its own words of
 * shared memory (no bank conflicts, no contention). The deposit accumulates
 * its tiles with such adds (two 32-bit adds per tap), so this is the peak of
 * its roofline. Runs on cuda_stream and synchronises it; writes adds per
 * second to *adds_per_s. MOND_EINVAL for other widths, MOND_ECUDA on a CUDA
 * error. */
int mond_pm_probe_smem_atomics(int bits, void* cuda_stream, double* adds_per_s);

/* Mass deposit for callers that cannot allocate device memory.
 * The paper has no counterpart; this entry point exists because some callers
 * cannot call cudaMalloc (a host framework that owns every device
 * allocation, a plug-in that must not grow the process's device footprint).
 * It computes the same density as mond_pm_deposit followed by
 * mond_pm_get_field(MOND_FIELD_RHO) -- bit for bit -- for N particles on an
 * n_f^3 periodic domain of pixel width s, writing rho_out (device float32,
 * n_f^3, caller-owned). Inputs are device arrays in the layout above.
 * It allocates nothing: its scratch (int64 accumulator of at most 128^3
 * cells, the lookup table for kernel widths up to 2 px, the ball of taps) is
 * held in fixed-size __device__ arrays that every GPU loading the library
 * keeps until the process exits (about 21 MiB per device).
 * Limits: 8 <= n_f <= 128, 0.75 <= kernel_width <= 2, N < 2^31; anything
 * else returns MOND_EINVAL with a message in mond_pm_last_error(NULL).
 * The first call on a device, and any call that changes kernel_width, sets
 * the scratch up and synchronises cuda_stream; make that call before any
 * stream capture. The set-up is tied to the device's current CUDA context:
 * after cudaDeviceReset the next call sets the scratch up again (and
 * synchronises). Every call shares the scratch: calls whose work overlaps on
 * the GPU race and give wrong results, so order them on one stream. On the
 * host, calls from several threads are serialised by a lock for as long as
 * they enqueue work; that does not order their GPU work. */
int mond_pm_deposit_noalloc(int32_t n_f, double s, double kernel_width, int64_t N, const int32_t* cell,
                            const float* offset, const float* mass, float* rho_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MOND_PM_H */
