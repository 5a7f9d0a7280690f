/*
 * liblbm -- D2Q9 stream-and-collide lattice Boltzmann method on one NVIDIA GB300 (sm_103a).
 *
 * The method is the one compared in Coreixas, Wissocq, Chopard & Latt, "Impact of
 * collision models on the physical properties and the stability of lattice Boltzmann
 * methods" (arXiv:2002.05265):
 *   f_i(x + xi_i, t + 1) = f*_i(x, t)                       (Eq. StreamCollide)
 * on a periodic nx x ny lattice (Sec. 5a), with the post-collision populations f* given by
 * one of the collision models of App. B, all built on the extended equilibrium of
 * Eq. extendedFeq (Sec. 4c).  Velocity index order (i: xi):
 *   0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).
 *
 * Conventions for every call below
 *   Return value   0 (LBM_OK) or a negative LBM_ERR_* code; lbm_last_error() gives detail.
 *   Pointers       Field arguments are plain pointers to dense row-major arrays
 *                  [ny][nx] (populations: [9][ny][nx]) of double.  They may point to
 *                  device memory (the call is then asynchronous on the context's stream
 *                  and the caller keeps the memory alive until the stream reaches it) or
 *                  to host memory, pageable or pinned (the call then copies through a
 *                  device staging buffer owned by the context and, for outputs, waits on
 *                  the stream before returning).  The library never keeps a caller
 *                  pointer after a call returns.
 *   Ownership      The context owns its two population buffers, staging and scratch
 *                  memory; lbm_destroy frees them.  Callers own every argument array.
 *   Streams        `cuda_stream` is a cudaStream_t (e.g. torch.cuda.current_stream().
 *                  cuda_stream); NULL means the legacy default stream.  All work of a
 *                  context is enqueued on that stream, in call order.
 *   Threads        A context must not be used from two host threads at once.
 */
#ifndef LBM_H
#define LBM_H

#ifdef __cplusplus
extern "C" {
#endif

/* Collision models (App. B).  PR is the standard regularized model = HM with
 * omega3 = omega4 = 1 (Sec. 5c, App. C); the omega3/omega4 passed with PR are ignored. */
typedef enum {
    LBM_BGK = 0,   /* f* = f - omega_nu (f - f^eq)                          (Sec. 1)        */
    LBM_RM  = 1,   /* raw moments relaxed by order                       (Eq. RMcoll)       */
    LBM_HM  = 2,   /* Hermite moments, then Eq. HM2RM_Q9                    (App. B)        */
    LBM_CM  = 3,   /* central moments, binomial back-transform              (App. B)        */
    LBM_CHM = 4,   /* central Hermite moments  (Eqs. CHpoly, CHMcoll, CHM2HM_Q9)            */
    LBM_K   = 5,   /* cumulants; C22 = K22 - (K20 K02 + 2 K11^2)/rho        (Sec. 4c)       */
    LBM_PR  = 6,   /* standard regularized (= REG-HM)                       (Sec. 5c)       */
    LBM_RR  = 7,   /* recursive regularized      (Eqs. HMColl_Q9, RRformulas_D2Q9)          */
    /* Two further readings of the cumulant model, whose definition the paper defers to an
     * external reference: the fourth-order central moment is rebuilt from the relaxed C22
     * with the product term of the PRE-collision second-order central moments (LBM_K_PRE) or
     * of their EQUILIBRIUM values (LBM_K_EQ), instead of the post-collision ones of LBM_K.
     * Linearly unstable at rest (Sec. 4b reports K so), but every simulation of Sec. 5b with
     * them blows up; kept to study that statement.  Same kernels as LBM_K. */
    LBM_K_PRE = 8,
    LBM_K_EQ  = 9
} lbm_model;

/* Population storage.  Every storage type holds the shifted populations
 * g_i = f_i - w_i rho0 (w_i the D2Q9 weights), rounded to nearest-even.  Collision
 * arithmetic is FP64 for LBM_F64 and FP32 for the others. */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16 = 2, LBM_BF16 = 3 } lbm_storage;

/* Relaxation frequencies per moment order (Sec. 4c): omega_nu for second order
 * (viscous, trace included), omega3 / omega4 for third / fourth order.  Each must lie in
 * (0, 2). */
typedef struct { double omega_nu, omega3, omega4; } lbm_rates;

enum {
    LBM_OK = 0,
    LBM_ERR_INVALID_ARG = -1,
    LBM_ERR_UNSUPPORTED = -2,   /* e.g. periodic = 0: the paper's domains are periodic (Sec. 5a) */
    LBM_ERR_CUDA = -3,
    LBM_ERR_BLOWUP = -4,        /* the blow-up criterion fired (see lbm_set_check)               */
    LBM_ERR_TIMEOUT = -5,       /* a bounded device-side wait gave up                            */
    LBM_ERR_NOMEM = -6
};

enum { LBM_PRESET_SRT = 0, LBM_PRESET_REG = 1 };

typedef struct lbm_ctx lbm_ctx;
typedef struct lbm_group lbm_group;

/* Sec. 4c: omega_nu = 1 / (nu / c_s^2 + 1/2) with c_s^2 = 1/3 (i.e. nu = c_s^2 (tau - 1/2)).
 * preset LBM_PRESET_SRT: omega3 = omega4 = omega_nu; LBM_PRESET_REG: omega3 = omega4 = 1.
 * Errors: nu <= 0 or non-finite, unknown preset, out == NULL -> LBM_ERR_INVALID_ARG. */
int lbm_rates_from_nu(double nu, int preset, lbm_rates* out);

/* Create a periodic nx x ny lattice context.
 *   periodic  must be 1 (LBM_ERR_UNSUPPORTED otherwise)
 *   model     lbm_model; storage lbm_storage
 *   eq_order  4 = extended equilibrium (Eq. extendedFeq, default for every model);
 *             3 = partial third-order equilibrium (Fig. 4: the extended one with its
 *                 fourth-order Hermite moment A^eq_22 set to zero) and
 *             2 = second-order equilibrium (Sec. 2; Hermite moments of order >= 3 set to
 *                 zero), both accepted for LBM_BGK only (LBM_ERR_UNSUPPORTED otherwise)
 *   rho0      reference density of the shift g = f - w rho0 (normally 1)
 * Errors: nx, ny < 3, nx*ny > 2^31, rates outside (0,2), unknown enums -> INVALID_ARG;
 *         device allocation failure -> LBM_ERR_NOMEM.  *out is NULL on error. */
int lbm_create(lbm_ctx** out, int nx, int ny, int periodic, int model, lbm_rates rates,
               int eq_order, int storage, double rho0, void* cuda_stream);

/* Release every device resource of the context (waits for its stream).  NULL is a no-op. */
void lbm_destroy(lbm_ctx* ctx);

/* Change the relaxation frequencies used by later steps (same validation as create). */
int lbm_set_rates(lbm_ctx* ctx, lbm_rates rates);

/* Change the storage shift to s_i = f^eq_i(rho0, u_ref) (extended equilibrium at a reference
 * velocity; the default u_ref = 0 gives s_i = w_i rho0) and re-encode the current state.
 * Choosing u_ref near the flow's mean velocity keeps the stored deviations small, which
 * cuts the rounding error of FP16/BF16 storage.  Not a concept of the paper: a storage
 * detail.  Errors: non-finite or |u_ref| >= 1 -> INVALID_ARG; eq_order 2 or 3 with u_ref != 0
 * -> UNSUPPORTED.  Waits on the context's stream. */
int lbm_set_shift_velocity(lbm_ctx* ctx, double ux_ref, double uy_ref);

/* f(x, 0) = f^eq(rho(x), u(x)) (Sec. 5a initial state; Eq. extendedFeq), computed in FP64
 * and rounded to the storage type; resets the step counter and the blow-up status. */
int lbm_init_equilibrium(lbm_ctx* ctx, const double* rho, const double* ux, const double* uy);

/* Advance n >= 0 time steps of Eq. StreamCollide (asynchronous).  Runs the blow-up check of
 * lbm_set_check at its cadence.  Returns LBM_OK once the work is enqueued; the blow-up
 * status is read with lbm_status. */
int lbm_step(lbm_ctx* ctx, long long n);

/* Macroscopic fields of the current pre-collision state f^n: rho = sum f_i,
 * u = sum xi_i f_i / rho, and the second-order raw moments Pi_ab = sum xi_a xi_b f_i
 * (Sec. 1; App. B).  Any output pointer may be NULL to skip it. */
int lbm_moments(lbm_ctx* ctx, double* rho, double* ux, double* uy,
                double* pxx, double* pxy, double* pyy);

/* FP64 global reductions of the current state (the diagnostics behind the blow-up
 * criterion of Sec. 5b), out[8] =
 *   [0] sum rho            [1] sum rho u_x          [2] sum rho u_y
 *   [3] sum rho |u|^2 / 2  [4] <|u|^2>              [5] <|u - uref|^2>
 *   [6] min rho            [7] number of nodes with non-finite rho or u
 * (<.> = mean over nodes; uref set by lbm_set_check).  Per-node values are computed in the
 * collision precision and summed in it over the four row segments a thread visits in a row
 * of its loop (8 nodes for FP64, 16 for FP32, 32 for 16-bit storage); those partial sums are
 * accumulated in FP64 in a fixed order (deterministic).  One launch: the last block to finish folds the per-block
 * partials, using a completion counter that the context owns and every launch leaves at zero.
 * Calls on one context must not overlap on the GPU (they share that scratch). */
int lbm_reduce(lbm_ctx* ctx, double* out8);

/* lbm_reduce without any allocation, for a population buffer the caller owns.
 *
 * The paper has no counterpart: this is a service for callers that cannot allocate device
 * memory when they need the diagnostics -- code that runs while another component is
 * capturing a CUDA graph in global mode (cudaMalloc is illegal there), code whose device
 * memory is owned entirely by a pool or caching allocator of the host application, and
 * latency-bound loops that must not call cudaMalloc/cudaFree (they synchronise the device).
 * lbm_reduce itself is unsuitable for them because lbm_create allocates.
 *
 *   populations  device pointer to one population buffer in the library's layout: nine
 *                planes g_i[y][x] (i in the index order above), row pitch `pitch` elements,
 *                plane = ny * pitch elements, element type given by `storage`, holding
 *                g_i = f_i - w_i rho0 with node x's population i at plane i, position
 *                x - xi_i (periodic), i.e. the state that the next pull step would read
 *   nx, ny       lattice size, 3 <= nx <= pitch, ny >= 3, nx * ny <= 2^31 (larger lattices
 *                are rejected with LBM_ERR_INVALID_ARG)
 *   uref_x/_y    reference velocity of out[5] only.  The buffer is always decoded with the
 *                w_i rho0 shift (storage-shift velocity zero): a buffer written by a
 *                context after lbm_set_shift_velocity with a non-zero velocity holds
 *                f_i - f^eq_i(rho0, u_ref) and is NOT supported -- its rho, momentum and
 *                blow-up figures would come out wrong without any error
 *   out8         device pointer to 8 doubles, same meaning as lbm_reduce (host pointers are
 *                rejected: copying them back would need staging memory)
 *   cuda_stream  stream to run on (NULL = legacy default stream); asynchronous
 * Both buffers must be on the current device (or managed memory).  Returns
 * LBM_ERR_INVALID_ARG for a null, misaligned or non-device pointer, a pointer to another
 * GPU's memory, an unknown storage or out-of-range sizes, LBM_ERR_CUDA if a launch fails.
 *
 * Scratch: the per-block partial sums go to one file-scope device array of 608 x 8 doubles
 * (38,912 bytes), which every GPU that loads the library holds until the process exits.  The
 * first call on each device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current; make that first call before any stream capture that could contain it.
 * The address is kept per device ordinal for the life of the process, so do not call this
 * after cudaDeviceReset on that device (the array of the new context has another address).
 * All calls share the array: calls that overlap on the GPU (e.g. on two streams at once)
 * race and give wrong results.  Each call rewrites every partial before reading it, so no
 * call depends on what the previous one left there.  No cudaMalloc, cudaFree or other
 * allocating routine is called. */
int lbm_reduce_noalloc(const void* populations, int storage, int nx, int ny, int pitch, double rho0,
                       double uref_x, double uref_y, double* out8, void* cuda_stream);

/* Halo exchange of a y-slab decomposition of one periodic lattice over several GPUs.  The
 * stream step of Eq. StreamCollide (Sec. 4a), f_i(x + xi_i, t + 1) = f*_i(x, t), crosses a
 * slab boundary only through the three populations with xi_y = +1 (i = 2, 5, 6) going up and
 * the three with xi_y = -1 (i = 4, 7, 8) going down.  A rank that owns rows y0 .. y1 - 1 of
 * the global lattice creates a context of ny = (y1 - y0) + 2 rows: local row r holds global
 * row y0 - 1 + r, and rows 0 and ny - 1 are ghost rows (a copy of the neighbours' boundary rows;
 * the context's own periodic wrap in y is never used for an owned row).  After every lbm_step
 * of one step the rank packs, sends, receives and unpacks:
 *   lbm_halo_pack(ctx, send_up, send_down): send_up <- planes 2, 5, 6 of local row ny - 2 (the
 *       post-collision populations its last own row emits upwards), send_down <- planes 4, 7, 8
 *       of local row 1.  Goes to the rank above / below.
 *   lbm_halo_unpack(ctx, from_below, from_above): from_below (the send_up of the rank below)
 *       -> planes 2, 5, 6 of ghost row 0; from_above (the send_down of the rank above) ->
 *       planes 4, 7, 8 of ghost row ny - 1.
 * Each message is 3 x nx raw storage elements ([3][nx], planes in the order listed, element
 * type of the context's storage, i.e. 3 * nx * {8, 4, 2} bytes), device pointers owned by the
 * caller; both calls are asynchronous on the context's stream and copy the stored (shifted)
 * values bit for bit, so every rank must use the same storage type and shift velocity.  After
 * an exchange, a step of the slab gives its own rows exactly what a step of the whole lattice
 * gives them.  The paper has no multi-GPU counterpart.  Errors: LBM_ERR_INVALID_ARG for a null
 * or host pointer, LBM_ERR_CUDA if the copy kernel fails to launch. */
int lbm_halo_pack(lbm_ctx* ctx, void* send_up, void* send_down);
int lbm_halo_unpack(lbm_ctx* ctx, const void* from_below, const void* from_above);

/* Canonical pre-collision populations f^n as FP64 [9][ny][nx] (unshifted), and the inverse
 * (values rounded to the storage type).  Used for checkpoint / resume and tests. */
int lbm_get_populations(lbm_ctx* ctx, double* f);
int lbm_set_populations(lbm_ctx* ctx, const double* f);

/* Blow-up check run by lbm_step every `every` steps (0 disables): the state is marked
 * blown up if any node has a non-finite rho or u, if min rho <= 0, or, when ke_ref > 0,
 * if <|u|^2> > ke_factor * ke_ref (Sec. 5b: <u^2>/u_0^2 < 1 with ke_ref = u_0^2,
 * ke_factor = 1).  uref is the reference velocity of out[5] in lbm_reduce. */
int lbm_set_check(lbm_ctx* ctx, long long every, double ke_ref, double ke_factor,
                  double uref_x, double uref_y);

/* Wait for the context's stream, then report: *status = LBM_OK, LBM_ERR_BLOWUP, or
 * LBM_ERR_TIMEOUT if a bulk-copy step kernel gave up waiting for its copies (a bounded wait
 * of about two seconds; it then stops advancing the lattice),
 * *blowup_step = first checked step at which the criterion fired (-1 if none),
 * *steps = steps taken since the last init.  Any pointer may be NULL. */
int lbm_status(lbm_ctx* ctx, int* status, long long* blowup_step, long long* steps);

/* Wait until all work enqueued on the context's stream has finished. */
int lbm_synchronize(lbm_ctx* ctx);

/* Grid geometry actually used: row pitch in elements (>= nx, multiple of 32), CUDA grid and
 * block sizes of the context's register-staged step kernel (the copy-engine kernel of
 * LBM_PATH_BULK / LBM_PATH_AUTO runs CTAs of 192, 320 or 576 threads, by kernel form, on every
 * resident slot). */
int lbm_get_layout(const lbm_ctx* ctx, int* pitch, int* grid, int* block);

/* Kernel family that advances a context (library design choice; the paper has no
 * counterpart).  Both compute the same pull stream-and-collide of Eq. StreamCollide:
 *   LBM_PATH_VECTOR  register-staged: each warp loads its nodes' nine pulled 16-byte vectors
 *                    itself (x-shifted elements by warp shuffles); any nx.
 *   LBM_PATH_BULK    copy-engine staged: cp.async.bulk copies each tile's nine pulled row
 *                    segments into a ring of `stages` (2-4; 0 = default) shared-memory stages
 *                    on mbarriers while 4-16 consumer warps (lbm_set_tile_form) collide
 *                    earlier tiles; needs nx * (bytes per population) to be a multiple of 16.
 *   LBM_PATH_AUTO    BULK where the row length allows it and a time step has at least one
 *                    tile per resident CTA, else VECTOR (the default).
 * Applies to the context's next lbm_step and to groups created afterwards.  Errors:
 * LBM_ERR_INVALID_ARG for an unknown path or stage count, LBM_ERR_UNSUPPORTED for BULK on a
 * lattice whose rows are not a multiple of 16 bytes. */
enum { LBM_PATH_AUTO = 0, LBM_PATH_VECTOR = 1, LBM_PATH_BULK = 2 };
int lbm_set_kernel_path(lbm_ctx* ctx, int path, int stages);

/* Launch shape of the copy-engine staged kernel (library design choice; the paper has no
 * counterpart; results are identical for every shape).  One launch may advance several time
 * steps: a tile of step s is copied once the rows it pulls from are complete in step s - 1
 * (row-completion counters in device memory, cooperative launch).
 *   steps_per_launch  time steps per launch; 0 = default (1 in the light and wide forms;
 *                     in the general form 16 with the wavefront order, else many when a
 *                     step has fewer than 64 tiles per CTA, 1 otherwise).
 *   order             LBM_ORDER_STEP: every tile of step s before those of step s + 1 (in
 *                     the CTAs' round-robin).  LBM_ORDER_WAVE (lattices of one geometry):
 *                     the steps of a launch interleave, a few rows behind one another, so
 *                     the intermediate states stay in the L2 and HBM sees about one read and
 *                     two writes per launch instead of one read and one write per step.
 *                     LBM_ORDER_BLOCK: step order with each CTA on a contiguous range of
 *                     tiles (so mostly on one lattice, one collision model, per step).
 *                     LBM_ORDER_AUTO: the wavefront for a single lattice whose buffers exceed
 *                     256 MB and that runs several steps per launch, else step order
 *                     (measured on GB300: the wavefront gains on single-model lattices of a
 *                     few GB, loses on mixed-model groups and with one-step launches).
 * Applies to the context's next lbm_step and to groups created afterwards (a group takes the
 * shape of its first context).  Errors: LBM_ERR_INVALID_ARG for a negative step count or an
 * unknown order. */
enum { LBM_ORDER_AUTO = 0, LBM_ORDER_STEP = 1, LBM_ORDER_WAVE = 2, LBM_ORDER_BLOCK = 3 };
int lbm_set_launch_shape(lbm_ctx* ctx, int steps_per_launch, int order);

/* Kernel form of the copy-engine staged kernel (library design choice; the paper has no
 * counterpart; results are identical for every form).  The forms differ in consumer warps per
 * CTA, CTAs per SM and the models compiled in:
 *   LBM_FORM_GENERAL  every model; 8 consumer warps, 2 CTAs per SM (FP64: 1).  Serves
 *                     multi-step launches (small lattices), where a CTA that waits on a row
 *                     counter leaves its SM to the other.
 *   LBM_FORM_LIGHT    BGK, RM, HM and PR only, FP32 / FP16 / BF16; FP32: 4 consumer warps,
 *                     2 CTAs per SM; 16-bit: 8 consumer warps, 1 CTA per SM, 8 nodes a thread.
 *   LBM_FORM_WIDE     every model, FP32 / FP16 / BF16; 16 consumer warps, 1 CTA per SM.
 *   LBM_FORM_AUTO     the default: the light form when every lattice of the group runs BGK, RM,
 *                     HM or PR in FP32 or FP16 storage, else the wide form, one time step per
 *                     launch, where a time step has at least 24 of the form's tiles per
 *                     resident CTA (or one step per launch is asked for with
 *                     lbm_set_launch_shape), except that a single lattice the general form
 *                     would advance in the wavefront order keeps the general form; the general
 *                     form otherwise (and for FP64).
 * Applies to the context's next lbm_step and to groups created afterwards (a group takes the
 * form of its first context when its lattices allow it, else LBM_FORM_AUTO).  Errors:
 * LBM_ERR_INVALID_ARG for an unknown form; LBM_ERR_UNSUPPORTED for LBM_FORM_LIGHT on another
 * model or on FP64 storage, or LBM_FORM_WIDE on FP64 storage. */
enum { LBM_FORM_AUTO = 0, LBM_FORM_GENERAL = 1, LBM_FORM_LIGHT = 2, LBM_FORM_WIDE = 3 };
int lbm_set_tile_form(lbm_ctx* ctx, int form);

/* Several contexts advanced together, one time step of each in turn (so a set of lattices
 * whose sum exceeds L2 streams from HBM as a single large one would), captured in CUDA
 * graphs of `graph_steps` steps (even, >= 2; 0 = no graphs).  Every context must use the
 * same stream.  Blow-up checks of each context run at their own cadence. */
int lbm_group_create(lbm_group** out, lbm_ctx* const* ctxs, int n, int graph_steps);
int lbm_group_step(lbm_group* g, long long nsteps);
void lbm_group_destroy(lbm_group* g);
/* Optional live timing of the graph replays with CUDA events on the group's stream:
 * enable, then read the summed duration (ms) of the replays, the number of lattice time
 * steps and the number of step-kernel launches they contained (waits on the stream).
 * A group of 2-16 contexts of one storage type advances all of them with one multi-lattice
 * launch per time step; otherwise each context gets its own launch. */
int lbm_group_set_timing(lbm_group* g, int enable);
int lbm_group_timing(lbm_group* g, double* replay_ms, long long* lattice_steps, long long* kernel_launches);
/* How the group is advanced (library design choice; the paper has no counterpart): *family =
 * LBM_PATH_BULK (copy-engine staged launches over all contexts), or LBM_PATH_VECTOR
 * (register-staged: one multi-lattice launch per step, or one launch per context and step);
 * for LBM_PATH_BULK, *form = LBM_FORM_GENERAL / LBM_FORM_LIGHT / LBM_FORM_WIDE, *steps_per_launch
 * the time steps of one launch, *tiles the tiles of one time step, *grid the resident CTAs a
 * launch may use and *block the CTA size; for LBM_PATH_VECTOR those four are 0 and *form is
 * LBM_FORM_AUTO.  Any pointer may be
 * NULL.  Errors: LBM_ERR_INVALID_ARG for a null group. */
int lbm_group_describe(const lbm_group* g, int* family, int* form, int* steps_per_launch, int* tiles, int* grid,
                       int* block);

/* Discrete adjoint of N steps (Eq. StreamCollide): lambda^n = dL/df^n runs backwards as
 *   lambda^n_j(x) = sum_i lambda^{n+1}_i(x + xi_i) dC_i/df_j(f^n(x))
 * (reverse streaming, then the transposed per-node collision Jacobian J of App. A,
 * Eq. Perturbed_Collision, taken at each node's own state), with the gradients
 *   dL/domega_k = sum_n sum_x sum_i lambda^{n+1}_i(x + xi_i) dC_i/domega_k   (FP64 sums),
 *   dL/du0_a(x) = sum_i lambda^0_i(x) df^eq_i/du_a(rho0(x), u0(x)).
 * The current state of the context is taken as f^0 = f^eq(rho0, u0) (call
 * lbm_init_equilibrium first); the call advances it to f^N.  Loss: 0 = misfit
 * L = 1/2 sum_x |u^N(x) - u*(x)|^2 with u* = (ux_target, uy_target) [ny][nx]; 1 = kinetic
 * energy L = 1/2 sum_x rho |u|^2 (targets ignored).  Memory: ceil(N/K) checkpoints plus K
 * recomputed states, K = checkpoint_every (0: ceil(sqrt(N))).  Outputs: grad_ux0/grad_uy0
 * [ny][nx], grad_rates3 = [dL/domega_nu, dL/domega3, dL/domega4] (zero for rates a model
 * does not use), *loss_out; any may be host or device pointers.  times_ms2 (host, optional):
 * [forward ms incl. checkpoints, backward ms incl. recomputation].
 * The storage shift of lbm_set_shift_velocity is honoured (a shift at the mean flow keeps the
 * FP32 trajectory, and so its gradient, closer to FP64).
 * Errors: storage other than FP64/FP32, or eq_order 2 or 3 -> UNSUPPORTED. */
int lbm_adjoint_run(lbm_ctx* ctx, long long nsteps, int loss, const double* ux_target, const double* uy_target,
                    int checkpoint_every, double* grad_ux0, double* grad_uy0, double* grad_rates3,
                    double* loss_out, double* times_ms2);

/* ---------------------------------------------------------------------------------------
 * Batched stability sweep: many independent periodic lattices of uneven size, each with its
 * own collision model, rates and blow-up detection, advanced by one persistent kernel launch
 * recorded in a CUDA graph (the numerical-stability study of Sec. 5b over (model, Ma, nu)).
 *
 * Blow-up criterion, evaluated every `check_every` steps on the pre-collision state with FP64
 * accumulation: any node with a non-finite rho or u, or min rho <= 0, or the perturbation
 * energy <|u - u_ref|^2> above `growth` times its value at the first check (values below
 * 1e-20 count as 1e-20), or, when ke_ref > 0, <|u|^2> > ke_factor * ke_ref (Sec. 5b with
 * ke_ref = u_0^2).  A blown-up instance stops; its step of detection is reported. */
typedef struct {
    int nx, ny;              /* lattice size (>= 3 each, nx * ny <= 2^31)                  */
    int model;               /* lbm_model                                                 */
    lbm_rates rates;         /* each in (0, 2); PR uses omega3 = omega4 = 1               */
    double ux_ref, uy_ref;   /* reference (mean-flow) velocity: of the perturbation energy
                                and of the storage shift g = f - f^eq(rho0, u_ref); |.| < 1 */
    double ke_ref, ke_factor;/* optional kinetic-energy criterion (ke_ref <= 0: off)      */
} lbm_instance_desc;

typedef struct lbm_batch lbm_batch;

/* Lay out n instances in one device slab (two buffers each, rows 32-byte aligned) for the
 * given storage type and shift density rho0.  Errors: invalid descriptors -> INVALID_ARG,
 * allocation failure -> NOMEM.  *out is NULL on error. */
int lbm_batch_create(lbm_batch** out, int n, const lbm_instance_desc* desc, int storage, double rho0,
                     void* cuda_stream);
void lbm_batch_destroy(lbm_batch* b);
/* Total number of nodes over all instances (the length of the concatenated fields). */
long long lbm_batch_nodes(const lbm_batch* b);
/* Equilibrium initial state of every instance (Eq. extendedFeq) from concatenated dense
 * fields: instance k's [ny][nx] block follows instance k-1's.  Host or device pointers.
 * Resets every instance's step counter and blow-up state.  Waits on the stream. */
int lbm_batch_init_equilibrium(lbm_batch* b, const double* rho, const double* ux, const double* uy);
/* Advance every live instance to `target_steps` total steps (asynchronous; one graph launch
 * of the persistent kernel).  growth > 1. */
int lbm_batch_run(lbm_batch* b, long long target_steps, int check_every, double growth);
/* Per-instance results (host arrays of n entries, any may be NULL; waits on the stream):
 * status 0 or LBM_ERR_BLOWUP, step of detection (-1 if none), steps taken, and diag4 =
 * n x [last <|u-u_ref|^2>, last <|u|^2>, last min rho, first-check <|u-u_ref|^2>]. */
int lbm_batch_status(lbm_batch* b, int* status, long long* blowup_step, long long* steps, double* diag4);
/* Canonical pre-collision populations of one instance as FP64 [9][ny][nx]. */
int lbm_batch_get_populations(lbm_batch* b, int index, double* f);
/* Kernel shape: `vec` x-nodes per thread and `block` threads per CTA.  autotune times every
 * instantiated shape for `trial_steps` steps from the current state (restoring the state
 * after each trial), keeps the fastest and reports it. */
int lbm_batch_set_shape(lbm_batch* b, int vec, int block);
int lbm_batch_get_shape(const lbm_batch* b, int* vec, int* block, int* grid);
int lbm_batch_autotune(lbm_batch* b, long long trial_steps, int check_every, int* vec, int* block,
                       double* best_ms);
const char* lbm_batch_last_error(const lbm_batch* b);

/* ---- Linear stability analysis (App. A) ---------------------------------------------
 * Growth rates of plane-wave perturbations of a uniform equilibrium state under the
 * stream-and-collide iteration: f'(x + xi_i, t + 1) = G f'(x, t), G = d f* / d f the Jacobian
 * of the collision map of `model` with `rates` at f = f^eq(rho, u) of equilibrium order
 * `eq_order` (as in lbm_create: 4 for every model, 2 or 3 for LBM_BGK only), and for
 * a wavenumber k the eigenproblem E^D(k) G A = exp(-i omega) A, E^D = diag(exp(-i xi_i . k))
 * (Eq. EigenvaluePbDiscrete).  G is the exact derivative of this library's own collision;
 * the eigenvalues come from a Hessenberg / shifted-QR solver in FP64 on the GPU.
 *   flows   device, nflows x 3 doubles (rho, ux, uy) of the base states
 *   k       device, nk x 2 doubles (kx, ky), radians per lattice spacing
 *   growth  device, nflows x nk doubles (row-major by flow): max over the nine modes of
 *           Im(omega) = ln |exp(-i omega)|
 *   eig     optional device, nflows x nk x 9 complex eigenvalues (re, im pairs)
 *   jac     optional device, nflows x 81 doubles: G row-major (G[i][j] = d f*_i / d f_j)
 * Synchronous on `stream`.  Errors: LBM_ERR_INVALID_ARG for an unknown model or equilibrium
 * order, a rate outside (0, 2), a host pointer or more than 2^31 flow x wavenumber pairs;
 * LBM_ERR_UNSUPPORTED for eq_order 2 or 3 with a model other than BGK; LBM_ERR_TIMEOUT if the QR
 * iteration did not converge for some matrix (its growth entry is NaN); LBM_ERR_CUDA /
 * LBM_ERR_NOMEM.  PR uses omega3 = omega4 = 1 whatever `rates` says. */
int lbm_lsa_growth(int model, lbm_rates rates, int eq_order, const double* flows, int nflows, const double* k, int nk,
                   double* growth, double* eig, double* jac, void* stream);

/* Text of the last error on this context (never NULL); lbm_error_string names a code. */
const char* lbm_last_error(const lbm_ctx* ctx);
const char* lbm_error_string(int code);

/* Library version string. */
const char* lbm_version(void);

/* Self-test of the FP32 reciprocal that forms u = j / rho (Sec. 1: u = (sum_i xi_i f_i) / rho)
 * in every FP32 kernel: the hardware approximation refined by one Newton-Raphson step.  The
 * paper has no counterpart (it fixes no arithmetic).  For n device floats x, writes the
 * library's reciprocal to approx[k] and the correctly rounded one (__frcp_rn) to rounded[k],
 * asynchronously on cuda_stream (NULL = legacy default stream).  All three are device
 * pointers to n floats, owned by the caller.  Documented behaviour: within one ulp of the
 * rounded value for finite non-zero x whose reciprocal is a normal number; NaN for x = 0,
 * +-inf and NaN (a node with such a density is non-finite either way).  Returns
 * LBM_ERR_INVALID_ARG for a null pointer or n < 0, LBM_ERR_CUDA if the launch fails. */
int lbm_selftest_recip(const float* x, float* approx, float* rounded, long long n, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
