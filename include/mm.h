/*
 * mm.h -- C ABI of the GB300 finite-difference micromagnetics library.
 *
 * The library evaluates the effective field of a finite-difference magnet and
 * advances the Landau-Lifshitz equation with adaptive Dormand-Prince RK45, as
 * described in "The design and verification of Mumax3" (Vansteenkiste et al.,
 * AIP Advances 4, 107133, 2014): Sec. II (grid, regions), Sec. III (torque and
 * effective-field terms), Sec. IV (time integration).
 *
 * Conventions for every entry point:
 *  - Return value: MM_OK (0) or a negative MM_ERR_* code.  mm_last_error()
 *    returns a NUL-terminated, thread-local message owned by the library that
 *    describes the last failure on the calling thread.
 *  - Units are SI: T, A/m, J/m, J/m^3, s, m.
 *  - Spatial arrays are cell-centred, x fastest: index (z*ny + y)*nx + x.
 *    Vector arrays are structure-of-arrays float32 [3][nz][ny][nx] (component
 *    planes x, y, z).  Byte maps (geometry, regions) are uint8 [nz][ny][nx].
 *  - Host pointers are read or written only during the call; the library never
 *    keeps them.  *_device variants take device pointers on the context's
 *    device; they are ordered on the context's stream and the call returns once
 *    the stream has finished with them.
 *  - A context owns all device memory it allocates and releases it in
 *    mm_destroy.  A context is not thread-safe: one thread at a time.
 */
#ifndef MM_H
#define MM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MM_OK = 0,
  MM_ERR_ARG = -1,          /* bad size, index, pointer or parameter           */
  MM_ERR_CUDA = -2,         /* a CUDA runtime call failed                      */
  MM_ERR_OOM = -3,          /* device allocation failed                        */
  MM_ERR_NONFINITE = -4,    /* NaN/Inf in the step error (and hence in m)      */
  MM_ERR_DT_UNDERFLOW = -5, /* a rejected step asked for dt below dt_min      */
  MM_ERR_TIMEOUT = -6,      /* a bounded device-side wait expired              */
  MM_ERR_STATE = -7         /* call out of order (e.g. stepping before set_m)  */
};

typedef struct mm_ctx mm_ctx;

/* Per-region material (Sec. II.A: 256-entry look-up tables by region index). */
typedef struct {
  double msat;      /* saturation magnetisation Msat (A/m); 0 = non-magnetic  */
  double aex;       /* exchange stiffness Aex (J/m), Eq. for B_exch           */
  double alpha;     /* damping, Eq. eqLLG                                     */
  double gamma_ll;  /* gyromagnetic ratio (rad/(T s)); 1.7595e11 by default    */
  double ku1, ku2;  /* uniaxial anisotropy constants (J/m^3), Sec. III.E      */
  double anis_u[3]; /* anisotropy axis (normalised by the library)            */
  double dind;      /* interfacial DMI constant D (J/m^2), Sec. III "Dzyaloshinskii-
                       Moriya interaction": B_DM = (2D/Msat)(dmz/dx, dmz/dy,
                       -dmx/dx - dmy/dy) by central differences; at a missing
                       neighbour (grid edge or vacuum) the Rohart boundary
                       conditions give a ghost value, used by exchange too.
                       D and Aex of the cell's own region; 0 = no DMI        */
  /* spin-transfer torques (Sec. III "Zhang-Li spin-transfer torque",
     "Slonczewski spin-transfer torque"; switched on by mm_enable_stt)       */
  double jcur[3];   /* current density j (A/m^2)                              */
  double xi;        /* Zhang-Li non-adiabaticity                              */
  double pol;       /* Slonczewski spin polarisation P                        */
  double lambda_sl; /* Slonczewski Lambda (>= 1 typical; 1 = angle-independent) */
  double eps_prime; /* Slonczewski secondary parameter eps'                   */
  double mp[3];     /* fixed-layer magnetisation direction (normalised)       */
  double tfree;     /* free-layer thickness d (m); 0 = no Slonczewski torque  */
} mm_material;

typedef struct {
  double total, demag, exch, anis, zeeman; /* J (total includes dmi)      */
  double m_avg[3];                         /* average m over magnetic cells */
  double dmi;                              /* J, -1/2 M.B_DM V summed       */
} mm_energies;

typedef struct {
  long long accepted;  /* accepted RK45 steps since creation                  */
  long long rejected;  /* rejected attempts                                   */
  long long evals;     /* torque evaluations (the paper's Neval)              */
  double last_err;     /* error estimate of the last attempt                  */
  double t, dt;        /* current time and the controller's proposed step     */
  long long launches;  /* kernels this context has launched (host count,      */
                       /* including graph nodes and no-op tail launches)      */
} mm_stats;

/* Message of the last failure on this thread ("" if none). */
const char* mm_last_error(void);

/* Grid of nx*ny*nz orthorhombic cells of dx*dy*dz metres (Sec. II.A; the
 * script calls setgridsize/setcellsize).  Allocates the state, computes the
 * demagnetising kernel on the device (Sec. III.B "Magnetostatic kernel") and
 * sets defaults: every cell in the geometry and in region 0, all materials
 * zero except gamma_ll = 1.7595e11, all terms enabled, MaxErr 1e-5, headroom
 * 0.8 (Sec. IV).  cuda_stream is a cudaStream_t on `device`, or NULL for a
 * stream owned by the context.  *out is NULL on failure. */
int mm_create(mm_ctx** out, int nx, int ny, int nz, double dx, double dy,
              double dz, int device, void* cuda_stream);
/* Releases the context and its device memory; NULL is accepted. */
int mm_destroy(mm_ctx* ctx);

/* Geometry mask (Sec. II.B): nonzero = magnet, 0 = vacuum.  NULL = all cells.
 * Vacuum cells carry m = 0, no torque, and drop out of the exchange sum. */
int mm_set_geometry(mm_ctx* ctx, const uint8_t* mask);
/* Region index per cell, 0..255 (Sec. II.A).  NULL = all region 0. */
int mm_set_regions(mm_ctx* ctx, const uint8_t* region);
/* Material of one region (0..255). */
int mm_set_region_material(mm_ctx* ctx, int region, const mm_material* mat);
/* Exchange scale S between two regions (Eq. for inter-region exchange,
 * symmetric, default 1). */
int mm_set_exchange_scale(mm_ctx* ctx, int r1, int r2, double S);
/* Applied field B_ext(region, t) = b0 + b1 sin(2 pi freq t + phase) (Sec. II.A
 * "Excitations": one function of time times a per-region profile).  region -1
 * sets every region.  b1 may be NULL (static field). */
int mm_set_bext(mm_ctx* ctx, int region, const double b0[3], const double b1[3]);
int mm_set_bext_timefn(mm_ctx* ctx, double freq, double phase);
/* Enables the demag, exchange, anisotropy and Zeeman terms and the precession
 * term of Eq. eqLLG (precession off = relaxation dynamics). */
int mm_enable_terms(mm_ctx* ctx, int demag, int exch, int anis, int zeeman,
                    int precession);

/* Periodic boundary conditions (Sec. III.B, "Periodic boundary
 * conditions"), macro geometry: px, py, pz images of the box on each side
 * along x, y, z (0 = open axis).  A source image contributes to a cell when
 * its offset along the periodic axis lies within -P n < D < P n (n cells);
 * the convolution along that axis becomes cyclic (no padding) and the
 * exchange and DMI stencils wrap around.  A periodic axis needs 1 cell or a
 * power of two >= 4 cells (else MM_ERR_ARG).  Rebuilds the demag kernel;
 * keeps m, t, the materials and the geometry mask.  (0, 0, 0) at creation. */
int mm_set_pbc(mm_ctx* ctx, int px, int py, int pz);

/* Spin-transfer torques added to dm/dt (off at creation): Zhang-Li,
 * dm/dt -= 1/(1+a^2)((1 + xi a) m x (m x h) + (xi - a) m x h) with
 * h = (u.grad) m, u = mu_B j / (2 e Msat (1 + xi^2)), central differences
 * (a missing neighbour is the cell itself; periodic axes wrap); Slonczewski,
 * dm/dt -= gamma beta/(1+a^2) ((eps - a eps') m x (m_P x m) - (eps' - a eps)
 * m x m_P), beta = j_z hbar / (Msat e d), eps = P L^2 / ((L^2+1) + (L^2-1)
 * m.m_P).  The printed torques are read in the sign convention of the LL
 * torque (dm/dt = -gamma tau).  A torque is active only in regions with
 * Msat > 0 and j != 0 (Slonczewski also needs tfree > 0 and j_z != 0); while
 * one is active the context steps with the general stage kernels. */
int mm_enable_stt(mm_ctx* ctx, int zhang_li, int slonczewski);

/* Reduced magnetisation m, float32 SoA [3][nz][ny][nx].  The library
 * normalises it per magnetic cell and zeroes it in vacuum.  Setting m
 * invalidates the cached first RK stage, unless the new m equals the current
 * one bit for bit (e.g. written back as read by mm_get_m): then the call
 * changes nothing. */
int mm_set_m(mm_ctx* ctx, const float* m);
int mm_get_m(mm_ctx* ctx, float* m);
int mm_set_m_device(mm_ctx* ctx, const float* dm);
int mm_get_m_device(mm_ctx* ctx, float* dm);

/* Adaptive step control (Sec. IV): MaxErr (default 1e-5), headroom (0.8),
 * initial step dt0 and the bounds dt_min, dt_max (s). */
int mm_set_solver(mm_ctx* ctx, double max_err, double headroom, double dt0,
                  double dt_min, double dt_max);
/* Replay mode: the next steps take exactly dts[0..n-1] and are all accepted
 * (the error is still computed and reported).  n = 0 returns to adaptive
 * stepping.  The array is copied. */
int mm_set_fixed_dt_sequence(mm_ctx* ctx, const double* dts, int n);

/* Failure detection (no counterpart in the paper): the row-stage kernels wait
 * for their tensor copies (TMA) on mbarriers, and every such wait is bounded.
 * `cycles` is the limit in SM clock cycles (default 2^30, about half a second
 * at 2.07 GHz); a wait that reaches it records MM_ERR_TIMEOUT in the device
 * state and the attempt is abandoned: the kernel first waits, with the
 * default limit, for its copies still in flight, then returns, and the later
 * kernels of the attempt skip their work.  mm_step / mm_run then return
 * MM_ERR_TIMEOUT with m, t and dt as they were before the abandoned attempt,
 * and the context stays usable.  0 gives up at the first wait without polling
 * (it exercises that error path; copies are never lost).  The limit is part of
 * the device state (kept in checkpoints).  MM_ERR_ARG if cycles < 0. */
int mm_set_wait_limit(mm_ctx* ctx, long long cycles);
int mm_get_wait_limit(mm_ctx* ctx, long long* cycles);

/* Integrator (Sec. IV "Dynamics"): MM_RK45, Dormand-Prince 5(4), 6 new
 * torque evaluations per attempt (default); MM_RK23, Bogacki-Shampine 3(2),
 * 3 per attempt, step factor exponent 1/3.  Both reuse the last stage as the
 * next first stage.  Switching keeps m, t, dt and the controller settings. */
enum { MM_RK45 = 0, MM_RK23 = 1 };
int mm_set_integrator(mm_ctx* ctx, int method);
int mm_get_integrator(mm_ctx* ctx, int* method);

/* Takes n accepted steps of the current integrator (the paper's steps(n)).
 * In replay mode takes min(n, remaining) steps. */
int mm_step(mm_ctx* ctx, int n);
/* Advances to t_end exactly (the paper's run(t)); the last step is shortened
 * to land on t_end.  Returns MM_OK immediately if t >= t_end. */
int mm_run(mm_ctx* ctx, double t_end);

int mm_get_time(mm_ctx* ctx, double* t, double* dt);
int mm_set_time(mm_ctx* ctx, double t, double dt);

/* Effective field, demag field and torque (dm/dt) at the current m and t,
 * float32 SoA [3][nz][ny][nx].  B_eff and the torque are zero in vacuum; the
 * demag field is the convolution result in every cell (stray field). */
int mm_get_beff(mm_ctx* ctx, float* b);
int mm_get_bdemag(mm_ctx* ctx, float* b);
int mm_get_torque(mm_ctx* ctx, float* tau);
/* Energies from the effective field with float64 accumulation (Sec. III:
 * -1/2 M.B_demag, -1/2 M.B_exch, -1/2 B(Ku1).M - 1/4 B(Ku2).M, -M.B_ext). */
int mm_get_energies(mm_ctx* ctx, mm_energies* e);
/* Maximum over the magnetic cells of |dm/dt| (rad/s) at the current m and t,
 * with the current precession switch (float32 torque, exact max). */
int mm_get_max_torque(mm_ctx* ctx, double* tau_max);
/* The paper's relax() (Sec. IV "Energy minimization"): with the precession
 * term off and the RK23 solver, advances in blocks of 3 accepted steps while
 * the total energy decreases, then while the maximum torque decreases; each
 * time the torque stops decreasing MaxErr is divided by sqrt(2), and the
 * level on which MaxErr first reaches 1e-9 is the last.  t advances as in a
 * run.  Afterwards the integrator, MaxErr and the precession switch are those
 * of before the call.  *steps_taken (may be NULL) receives the accepted steps.
 * MM_ERR_TIMEOUT if a further block would exceed max_steps (the state reached
 * so far is kept); MM_ERR_STATE in replay or surrogate mode or before set_m. */
int mm_relax(mm_ctx* ctx, long long max_steps, long long* steps_taken);
int mm_get_stats(mm_ctx* ctx, mm_stats* s);
/* Sizes of the accepted steps since creation (up to `max` of them, oldest
 * first; the library keeps the first 1<<20); *n receives the count copied. */
int mm_get_dt_history(mm_ctx* ctx, double* dts, int max, int* n);

/* Checkpoint: the full integrator state (m, the cached first stage, t, dt,
 * controller settings, counters) as an opaque byte blob; resume is bit-exact.
 * A replay sequence (mm_set_fixed_dt_sequence) is not part of it: restoring
 * returns to adaptive stepping.  The blob is tied to the grid size. */
size_t mm_state_bytes(mm_ctx* ctx);
int mm_get_state(mm_ctx* ctx, void* buf, size_t bytes);
int mm_set_state(mm_ctx* ctx, const void* buf, size_t bytes);

/* Cell-averaged demagnetising tensor (Sec. III.B "Magnetostatic kernel") of
 * two dx*dy*dz cells at n integer offsets offsets[3i..3i+2] = (X, Y, Z) in
 * cells, computed on `device` in float64: out[6i..6i+5] = Nxx, Nyy, Nzz, Nxy,
 * Nxz, Nyz with the positive convention (self term of a cube 1/3,
 * B = -mu0 N M).  Host arrays. */
int mm_demag_tensor(int device, double dx, double dy, double dz, int n,
                    const int32_t* offsets, double* out);

/* Demagnetising field alone (Sec. III.B convolution) of the magnetisation
 * m (device pointer, float32 SoA [3][nz][ny][nx], read as Msat m with the
 * context's regions and geometry) into b (device pointer, same layout).
 * Ordered on the context's stream; returns after the stream has finished. */
int mm_demag_apply(mm_ctx* ctx, const float* m, float* b);

/* Demagnetising field B (T) of a magnetisation M = Msat m (A/m) on an
 * nx*ny*nz grid of dx*dy*dz cells, without allocating device memory.  For
 * callers that cannot call cudaMalloc: frameworks whose device memory must all
 * come from their own pool, applications that forbid device allocation after
 * start-up, real-time loops that must not touch the allocator.  The paper has
 * no counterpart; the arithmetic is the convolution of mm_demag_apply with a
 * kernel computed as in mm_create, redone on every call (a context is faster
 * for repeated use on one grid).
 *  - M, B: device pointers on the current device, float32 SoA [3][nz][ny][nx];
 *    the caller owns them.  stream: a cudaStream_t, or NULL.
 *  - Scratch: one static device array of 32 MiB (33 554 432 bytes) per GPU
 *    that loads the library, held until the process exits.  A grid needs
 *    16 KB of tables + 2 bytes per cell + the float32 kernel octant (24 B per
 *    point of (px/2+1)(py/2+1)(pz/2+1)) + the spectrum (24 B per point of
 *    nz * (py if nz > 1 else ny) * hxs, hxs = px/2+1 rounded up to 8) + two
 *    float64 precompute areas (48 B per point of the largest of n,
 *    (px/2+1) ny nz, (px/2+1)(py/2+1) nz and the octant) + a small table,
 *    each rounded up to 256 bytes (px, py, pz: the padded sizes, the power of
 *    two >= 2n - 1).  So 512x256x1, 384x256x1 and 64x64x32 fit, while
 *    512x512x1, 1024x256x1, 128x64x32 and 128x128x16 do not.  A grid that
 *    does not fit is rejected with MM_ERR_ARG and a message giving the bytes
 *    it needs, before any device call.
 *  - The first call on a device (and the first after that device's context
 *    was re-created) looks up the array's device address with that device
 *    current (cudaGetSymbolAddress); make that first call before any stream
 *    capture.
 *  - Every call uses the same array and leaves its contents behind (each call
 *    re-initialises what it reads); calls that overlap on the GPU (other
 *    streams, other threads) race.  The call synchronises `stream` before it
 *    returns.  It calls no cudaMalloc, cudaFree or allocating library
 *    routine. */
int mm_demag_field_noalloc(int nx, int ny, int nz, double dx, double dy, double dz,
                           const float* M, float* B, void* stream);

/* Blocks until the context's stream is idle. */
int mm_sync(mm_ctx* ctx);

/* Measurement of the stepping kernels (no counterpart in the paper).  Runs
 * `attempts` RK45 attempts from the current state, as mm_step(attempts)
 * would (each accepted or rejected by the controller), launched one kernel
 * at a time with a CUDA event recorded on the context's stream after each
 * launch instead of replaying the attempt's graph.  For each launch position
 * of one attempt (*n_out of them, at most max) it writes the kernel kind
 * (kinds[i]: 0 stage-input prep, 1 (y, z) demag convolution cluster kernel,
 * 2 row-stage kernel: x transforms, field, torque, stage update; with the
 * three-kernel (y, z) path 3 y forward, 4 column kernel: z forward, kernel
 * product, z inverse, 5 y inverse; 6 earlier-stage sums of the next row
 * kernel) and its mean duration over the attempts in microseconds (us[i]).
 * The events keep each kernel from overlapping its neighbour (no
 * programmatic-dependent-launch overlap; the earlier-stage sums, a branch
 * beside the (y, z) part in the graph, run in line here), so the sum can
 * exceed the graph's time per attempt.  L2 is not
 * flushed between launches.  MM_ERR_STATE before set_m and unless the context
 * steps with the fused row-stage kernels (RK45, exact demag, no periodic x
 * axis, no spin-transfer torque); the controller's errors as mm_step. */
int mm_profile_attempts(mm_ctx* ctx, int attempts, int max, int* kinds, double* us, int* n_out);

/* How the (y, z) part of the demag convolution (Sec. III.B) runs on a grid
 * with the fused spectrum layout (no counterpart in the paper; both compute
 * the same convolution, up to float32 rounding): which = 0 the grid's
 * default (2 where available, else 1), 1 one thread-block cluster per kx
 * plane (the (ky, kz) plane split into frequency residue classes across the
 * cluster's blocks, summed through distributed shared memory), 2 the
 * register-resident kernels: on 3-D grids three kernels over a y-transformed
 * buffer of 24 B per (kx, z, ky) point (y forward; per (kx, ky) column z
 * forward, kernel product and z inverse; y inverse), on 2-D grids one kernel
 * per kx plane (y forward, kernel product, y inverse).  2 needs open y and z
 * axes and, in 3-D, py >= 32 and 16 <= pz <= 64, in 2-D (one layer) py of
 * 128, 256 or 512 (MM_ERR_ARG otherwise).  *active (may be NULL) receives the
 * kernels in use: 1 or 2, or 0 on a grid without the fused layout.  The
 * stepping graph is captured again at the next step. */
int mm_set_yz_kernels(mm_ctx* ctx, int which, int* active);

/* FP32 fused multiply-add throughput of `device` (no counterpart in the
 * paper; the ALU roof of the convolution's arithmetic): a kernel of
 * independent FMA chains on every SM, timed with CUDA events on an internal
 * stream (best of `reps` launches after one warm-up).  *tflops receives
 * 2 x FMAs / time in TFLOP/s; *sm_count the device's multiprocessors and
 * *clock_mhz its maximum SM clock (may be NULL).  MM_ERR_ARG for reps < 1. */
int mm_fp32_peak(int device, int reps, double* tflops, int* sm_count, int* clock_mhz);

/* ---- Learned demag surrogate ----------------------------------------------
 * A Fourier-neural-operator approximation of the demag field of a 2-D film
 * (the learned form of the convolution of Sec. III.B; the paper has none).
 * u = Msat m / ms_ref -> y = B_demag / (mu0 ms_ref):
 *   v_0 = P u + p;  v_{l+1} = act(W_l v_l + b_l + K_l v_l);  y = Q v_L + q,
 * act = GELU (none after the last layer), K_l the spectral convolution
 * truncated to kx < modes_x and ky in {0..modes_y-1} U {H-modes_y..H-1},
 * written with explicit partial DFTs (Re of the inverse).  The x-direction
 * partial DFTs and the gradient products run on the bfloat16 tensor cores
 * with float32 accumulation; for widths 4, 8, 16 and 32 the forward pass's
 * pointwise products (lift, W_l v + b_l with the inverse x partial DFT and
 * the GELU, projection) run in float32, fused per layer.  The forward pass
 * is deterministic (fixed summation orders).  Parameters are float32 (Adam),
 * flat in the order P, p, {W_l, b_l, R_l}, Q, q with R_l complex
 * [width][width][2 modes_y][modes_x] as (re, im) pairs.
 * Loss: sum |yhat - y|^2 / sum |y|^2 over a batch. */
typedef struct mm_fno mm_fno;
typedef struct {
  int width, layers, modes_x, modes_y;
  int max_batch;               /* samples per forward/backward call        */
  unsigned long long seed;     /* initial parameters                       */
} mm_fno_cfg;
/* ny = H, nx = W.  MM_ERR_ARG unless H, W >= 2, width, layers, max_batch >= 1,
 * modes_x <= W / 2 and 2 modes_y <= H (checked before any device call);
 * MM_ERR_OOM / MM_ERR_CUDA from the allocations.  cuda_stream NULL: the
 * network creates its own stream. */
int mm_fno_create(mm_fno** out, int ny, int nx, const mm_fno_cfg* cfg, int device, void* cuda_stream);
int mm_fno_destroy(mm_fno* f);
long long mm_fno_param_count(mm_fno* f);
int mm_fno_get_params(mm_fno* f, float* host, long long n);
int mm_fno_set_params(mm_fno* f, const float* host, long long n);   /* resets Adam */
/* Device pointers, float32 [S][3][ny][nx], 1 <= S <= max_batch (else
 * MM_ERR_ARG); returns after the network's stream is idle. */
int mm_fno_forward(mm_fno* f, const float* u, float* y, int S);
/* Loss and its gradient (host array of param_count floats, may be NULL). */
int mm_fno_grad(mm_fno* f, const float* u, const float* y, int S, float* grad_host, double* loss);
/* One Adam step (beta 0.9, 0.999) on the batch; returns the batch loss. */
int mm_fno_train_step(mm_fno* f, const float* u, const float* y, int S, double lr, double* loss);
/* Trains `net` on n_pairs (m, B_demag) pairs taken from the context's own
 * exact trajectories: traj_len pairs per trajectory, steps_between exact RK45
 * steps apart, each trajectory from m uniform on the sphere per cell under a
 * static field of uniform direction and magnitude U[0, field_max]; then
 * `epochs` passes of Adam over shuffled batches.  The context's m, time and
 * fields are restored.  *final_loss receives the last batch loss. */
int mm_surrogate_train(mm_ctx* ctx, mm_fno* net, double ms_ref, int n_pairs, int traj_len,
                       int steps_between, double field_max, int epochs, int batch, double lr,
                       unsigned long long seed, double* final_loss);
/* Uses `net` for the demag field inside every RK stage (net NULL: exact
 * convolution).  Every check_every accepted steps the exact convolution
 * judges the surrogate at the current m; once the relative L2 field error
 * exceeds fallback_rel_err the context returns to the exact path for good.
 * Only mm_step is available in this mode. */
int mm_set_demag_surrogate(mm_ctx* ctx, mm_fno* net, double ms_ref, int check_every,
                           double fallback_rel_err);
int mm_get_surrogate_stats(mm_ctx* ctx, long long* steps_with_surrogate, long long* checks,
                           long long* fallbacks, double* last_rel_err, int* active);

/* ---- Batched simulations --------------------------------------------------
 * Many independent simulations of uneven grid sizes advanced together, each
 * with its own adaptive Dormand-Prince step (Sec. IV) and its own material and
 * static applied field (demag + exchange + Zeeman, every cell magnetic, one
 * material per instance).  Instances of the same grid and cell size share one
 * demag kernel.  A run is one CUDA graph launch that repeats batched RK45
 * attempts on the device until every instance reaches t_end. */
typedef struct mm_batch mm_batch;
typedef struct {
  int nx, ny, nz;           /* grid (nx >= 17; the padded (y, z) plane of   */
  double dx, dy, dz;        /* one grid must fit one thread-block cluster)  */
  double msat, aex, alpha;  /* material (A/m, J/m, -)                       */
  double gamma_ll;          /* rad/(T s); <= 0 means 1.7595e11              */
  double bext[3];           /* static applied field (T)                     */
} mm_instance_spec;

/* Creates n instances (specs copied); m starts at zero: set it with
 * mm_batch_set_m before running.  Defaults as in mm_create. */
int mm_batch_create(mm_batch** out, int n, const mm_instance_spec* specs, int device,
                    void* cuda_stream);
int mm_batch_destroy(mm_batch* b);
/* m of instance i, float32 SoA [3][nz][ny][nx] of that instance (host);
 * normalised per cell on upload. */
int mm_batch_set_m(mm_batch* b, int i, const float* m);
int mm_batch_get_m(mm_batch* b, int i, float* m);
/* Step control of every instance (as mm_set_solver). */
int mm_batch_set_solver(mm_batch* b, double max_err, double headroom, double dt0,
                        double dt_min, double dt_max);
/* Advances every instance to t_end (last step shortened to land on it). */
int mm_batch_run(mm_batch* b, double t_end);
/* Counters of instance i; returns that instance's status (MM_OK or the error
 * that stopped it). */
int mm_batch_get_stats(mm_batch* b, int i, mm_stats* s);
/* Accepted step sizes of instance i (the first 4096), as mm_get_dt_history. */
int mm_batch_get_dt_history(mm_batch* b, int i, double* dts, int max, int* n);
/* Number of shape classes (distinct grids) in the batch. */
int mm_batch_num_classes(mm_batch* b);
/* FFT tiles of class c, picked at creation by timing every candidate of the
 * class's convolution (no counterpart in the paper): info = {nx, ny, nz,
 * instances, cly, clz, xrows} (residue split of the (y, z) transform across a
 * cluster of cly*clz blocks; rows per block of the x-row kernels), *conv_us
 * (may be NULL) = the chosen convolution's time for all the class's
 * instances in microseconds. */
int mm_batch_class_info(mm_batch* b, int c, int info[7], double* conv_us);
/* Pins the FFT tiles of class c instead of the autotuner's choice (for
 * reproducible timings and tests): (cly, clz) must be one of the residue
 * splits the class's fused plan offers (each of 1 or 2, py/cly >= ny,
 * pz/clz >= nz, at most 4096 points per block) and xrows one of the offered
 * x-row block sizes (the default rule, half or twice it); MM_ERR_ARG
 * otherwise.  Takes effect at the next mm_batch_run (the run's graph is
 * captured again); the result differs from the autotuned tiles' only by
 * float32 rounding. */
int mm_batch_set_tiles(mm_batch* b, int c, int cly, int clz, int xrows);

#ifdef __cplusplus
}
#endif
#endif /* MM_H */
