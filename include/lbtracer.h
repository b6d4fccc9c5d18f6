/*
 * lbtracer.h -- C ABI of the GB300 tracer-box lattice Boltzmann library.
 *
 * The library advances many small lattice Boltzmann boxes, each of which
 * follows one Lagrangian tracer of a coarse turbulent flow, as in Lee,
 * Duenweg and Schumacher, "Multiscale modelling strategy using the lattice
 * Boltzmann method for polymer dynamics in a turbulent flow" (arXiv:0809.4958):
 *
 *   - D3Q19 lattice (Sec. 3), BGK collision with relaxation time tau
 *     (the paper does not print the operator; BGK is the reading),
 *     viscosity nu = (tau - 1/2) / 3 in lattice units;
 *   - initial condition: local equilibrium with the prescribed velocity on
 *     every site at t = 0 (Sec. 2);
 *   - boundary condition: for t > 0 the outer site layer is set to the local
 *     equilibrium of the prescribed boundary velocity (Sec. 2), interpolated
 *     in time between coarse samples (Sec. 3, after Eq. 1);
 *   - a bead-spring chain coupled to the fluid through a Stokes friction
 *     coefficient (Sec. 1, Ahlrichs-Duenweg hybrid method) with its centre of
 *     mass pinned at the tracer, i.e. the box centre (Sec. 2).  The chain is
 *     the Kremer-Grest model of that method: FENE bonds plus WCA repulsion.
 *
 * Conventions
 *   Lattice units throughout (spacing 1, time step 1, reference density 1).
 *   A box has E sites per axis (E a multiple of 8, 8 <= E <= 1024); site
 *   (x, y, z) is stored at linear index (z*E + y)*E + x (x fastest).
 *   Population order: rest; +x, -x, +y, -y, +z, -z; then (1,1,0), (-1,-1,0),
 *   (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1), (0,1,1),
 *   (0,-1,-1), (0,1,-1), (0,-1,1).
 *   Face order: x-, x+, y-, y+, z-, z+.  In-face coordinates (p, q) are
 *   (y, z) on x faces, (x, z) on y faces, (x, y) on z faces; a face array is
 *   [3 components][q][p].  A site on several velocity faces belongs to the
 *   first of them in face order.
 *   "real" below is double for LB_STORE_F64 and float for every other storage.
 *
 * Memory ownership
 *   The library never allocates device memory.  lb_plan reports the size of
 *   one device arena; the caller allocates it (for example as a torch tensor),
 *   keeps it alive until lb_destroy, and passes it to lb_create.  Every other
 *   pointer argument is borrowed for the duration of the call (host or device
 *   memory, told apart with cudaPointerGetAttributes) unless stated otherwise.
 *   All work is enqueued on the caller's CUDA stream given to lb_create; calls
 *   return after enqueueing except those documented as synchronising.
 *
 * Errors
 *   Every function returns LB_OK (0) or an LB_ERR_* code; lb_last_error gives
 *   a message.  Kernels never trap: a box whose chain breaks a rule (bond at
 *   the FENE limit, bead stencil leaving the interior) or whose state turns
 *   non-finite gets a device status word and is frozen (its state stops
 *   changing); the code is returned by the next synchronising call.
 */
#ifndef LBTRACER_H
#define LBTRACER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define LB_OK 0
#define LB_ERR_ARG 1        /* bad argument: shape, tau <= 1/2, E not a multiple of 8, null pointer */
#define LB_ERR_CUDA 2       /* a CUDA runtime call failed */
#define LB_ERR_FENE 3       /* a bond reached the FENE maximum extension R0 */
#define LB_ERR_BEAD_OOB 4   /* a bead's interpolation stencil left the box interior */
#define LB_ERR_NONFINITE 5  /* a site density met while stepping, or a mass or momentum sum, is not finite or <= 0 */
#define LB_ERR_TIMEOUT 6    /* a bounded wait expired: for the stream on the host, or a device pipeline wait */
#define LB_ERR_STATE 7      /* call out of order (e.g. stepping past the last boundary sample) */
#define LB_ERR_SIZE 8       /* arena too small for the plan */
#define LB_ERR_CHAIN 9      /* a bead has more WCA neighbours than the per-bead list holds (48) */

/* ---- population storage (one per context) ---- */
#define LB_STORE_F64 0      /* f_i - w_i in FP64, FP64 arithmetic */
#define LB_STORE_F32 1      /* f_i - w_i in FP32, FP32 arithmetic */
#define LB_STORE_F16DEV 2   /* f_i - w_i in IEEE binary16 (round to nearest even), FP32 arithmetic */
#define LB_STORE_BF16DEV 3  /* f_i - w_i in bfloat16 (round to nearest even), FP32 arithmetic */

/* ---- face modes (both faces of an axis must agree) ---- */
#define LB_FACE_VELOCITY 0  /* outer layer set to the equilibrium of the boundary velocity */
#define LB_FACE_PERIODIC 1

/* ---- time interpolation of the coarse boundary samples ---- */
#define LB_TIME_LINEAR 0    /* linear between samples j and j+1 (the paper's form) */
#define LB_TIME_HERMITE 1   /* cubic Hermite, Catmull-Rom tangents, one-sided on the first interval */
#define LB_TIME_MLP 2       /* Hermite plus the residual of the learned upsampler (lb_mlp_bind), K = 8 or 16 */

/* ---- fields for lb_read_fields ---- */
#define LB_FIELD_RHO 0      /* real [E^3] density */
#define LB_FIELD_U 1        /* real [3][E^3] velocity */
#define LB_FIELD_DEV 2      /* real [19][E^3] stored populations minus weights, f_i - w_i */
#define LB_FIELD_CHAIN 3    /* double [2][nbeads][3]: positions then velocities */
#define LB_FIELD_ASYNC 0x100 /* OR-ed into `what`: enqueue the read-out only, no wait, no status check */

#define LB_ALL_BOXES (-1)

/*
 * Coarse grid (Sec. 3: the DNS grid spacing is z LB spacings).  Boundary
 * samples and the initial field are given on a grid of Ec points per axis,
 * point P at site P z, Ec = ceil((E - 1)/z) + 1 (Ec = E when z <= 1); when z
 * does not divide E - 1 the last coarse cell reaches past the box.  A face
 * sample holds the face plane (site 0 or E - 1 along the normal) at the
 * coarse in-face points.  The boundary velocity of a face site is the
 * bilinear interpolation, within the face, of the time-interpolated
 * velocities at the four surrounding coarse points; the initial field is
 * trilinear between the eight surrounding coarse points.  1 <= z <= E - 1;
 * boxes with LB_TIME_MLP take z <= 1.
 */
typedef struct lb_box_desc {
    int32_t E;             /* sites per axis, multiple of 8 */
    int32_t face_mode[6];  /* LB_FACE_* per face, x-, x+, y-, y+, z-, z+ */
    int32_t time_interp;   /* LB_TIME_* */
    int32_t K;             /* LB steps per coarse sample interval, >= 1 */
    int32_t nbeads;        /* capacity for the chain of this box (0 = no chain), <= 256 */
    int32_t zoom;          /* z = coarse grid spacing in sites (Sec. 2-3); 0 or 1: samples on every site */
    int32_t frame_accel;   /* 1: the box also takes frame-acceleration samples (lb_set_frame_accel); 0 */
    double tau;            /* BGK relaxation time, > 1/2 */
    double rho_b;          /* density of the boundary equilibrium (1.0) */
    double body_accel[3];  /* uniform body acceleration a; force density rho a (Guo forcing) */
} lb_box_desc;

typedef struct lb_chain_desc {
    int32_t nbeads;        /* beads in the chain, 1 .. capacity given in lb_box_desc */
    int32_t n_md;          /* MD substeps per LB step, >= 1 */
    int32_t pin_com;       /* 0 off, 1 pin the centre of mass at the box centre, 2 also zero its velocity */
    int32_t reserved;
    double k_fene;         /* FENE spring constant k */
    double R0;             /* FENE maximum bond length */
    double zeta;           /* bead friction coefficient (Stokes friction of the coupling) */
    double mass;           /* bead mass */
    double kT;             /* temperature of the bead noise (0 = none) */
    double eps;            /* WCA repulsion strength between all bead pairs (0 = FENE bonds only) */
    double sigma;          /* WCA length; the repulsion acts below 2^(1/6) sigma */
    double f_ext[3];       /* constant external force on every bead */
    uint64_t seed;         /* Philox key of the bead noise */
} lb_chain_desc;

typedef struct lb_ctx lb_ctx;

/*
 * lb_plan -- size of the device arena for a context of tracer boxes (Sec. 2:
 * one fine lattice Boltzmann box per Lagrangian tracer, each fed by the
 * coarse flow around it; Sec. 3: the paper follows 100 tracers).
 *   boxes[nboxes]: box descriptions (host).  storage: LB_STORE_*.
 *   ring_slots: coarse samples the boundary ring holds (0 = 4, at most 4096).
 *   Four slots cover one step at a time; a captured graph of G steps needs
 *   G / K + 4 slots so that all its samples can be pushed before it runs.
 *   *arena_bytes receives the number of bytes the caller must allocate
 *   (device memory, 256-byte aligned).
 *   Returns LB_ERR_ARG for an invalid description.
 */
int32_t lb_plan(const lb_box_desc* boxes, int32_t nboxes, int32_t storage, int32_t ring_slots, size_t* arena_bytes);

/*
 * lb_create -- build a context over a caller-owned arena: the boxes of
 * lb_plan, each to be given its initial condition (lb_init), its boundary
 * samples (lb_set_boundary) and its chain (chain_couple) in the order of
 * Sec. 2 before it is stepped.
 *   arena: device pointer to at least the lb_plan size; borrowed until lb_destroy.
 *   stream: the cudaStream_t every later call enqueues on (NULL = legacy default stream).
 *   The library creates one private side stream and a few events for
 *   concurrency between the bead kernel and the stream-collide kernel.
 *   Populations are left uninitialised until lb_init.
 */
int32_t lb_create(const lb_box_desc* boxes, int32_t nboxes, int32_t storage, int32_t ring_slots, void* arena,
                  size_t arena_bytes, void* stream, lb_ctx** out);

/* lb_destroy -- wait for the stream, release the host context, events, side
 * stream and any captured graph.  Does not free the arena. */
int32_t lb_destroy(lb_ctx* ctx);

/*
 * lb_init -- initial condition (Sec. 2): every site of the box gets the local
 * equilibrium with density 1 and velocity u0.
 *   u0: real [3][Ec^3] on the coarse grid of the box ([3][E^3] for zoom <= 1),
 *   host or device.  A host array is staged through the
 *   box's second population buffer.  A one-box context may be re-initialised
 *   at any time (step counter and boundary ring restart at 0); the boxes of a
 *   multi-box context are initialised before the first lb_step
 *   (LB_ERR_STATE otherwise).
 */
int32_t lb_init(lb_ctx* ctx, int32_t box, const void* u0);

/*
 * lb_set_boundary -- push coarse boundary sample j (taken at t = j K) into
 * the ring of the box (Sec. 3: boundary velocities interpolated in
 * time between the samples).
 *   face_u: real [6][3][Ec][Ec] for one box (the coarse face points; Ec = E
 *   for zoom <= 1), or, with box == LB_ALL_BOXES, the arrays of all boxes back
 *   to back in box order; host or device.
 *   Samples must be pushed in order 0, 1, 2, ...; sample j may be pushed
 *   once no step still to be enqueued needs sample j - ring_slots.
 *   The copy is enqueued on the context stream (pinned host memory keeps it
 *   asynchronous).  A zoomed box's sample is interpolated bilinearly onto
 *   its face sites as it is pushed (Sec. 3: bilinear in space, interpolated
 *   in time; both are linear, so a step then interpolates in time only).
 */
int32_t lb_set_boundary(lb_ctx* ctx, int32_t box, int64_t sample_index, const void* face_u);

/*
 * lb_set_frame_accel -- push frame-acceleration sample j (taken at t = j K)
 * of a box created with frame_accel = 1 (Sec. 2: in the co-moving frame of
 * the tracer the flow w = u - v(t) feels the extra force density
 * rho (-dv/dt)).  a: host, 3 doubles, the acceleration -dv/dt in lattice
 * units at t = jK.  Step n -> n+1 applies the body acceleration
 * body_accel + a(t_n), a(t_n) linear between samples j = n / K and j + 1
 * (both must have been pushed; they share the boundary ring's slots, so the
 * same ordering rule as lb_set_boundary holds).  Enqueued on the context
 * stream.  LB_ERR_ARG for a box without frame_accel.
 */
int32_t lb_set_frame_accel(lb_ctx* ctx, int32_t box, int64_t sample_index, const double* a);

/*
 * chain_couple -- place the bead-spring chain of a box (Sec. 1 and 2).
 *   pos0, vel0: double [nbeads][3], host or device (vel0 may be NULL = 0).
 *   Bead positions are in lattice units; on a velocity axis the bead's
 *   trilinear stencil must stay within sites 1 .. E-2.
 */
int32_t chain_couple(lb_ctx* ctx, int32_t box, const lb_chain_desc* desc, const double* pos0,
                     const double* vel0);

/*
 * lb_step -- enqueue nsteps lattice Boltzmann steps for every box.  Each
 * step n -> n+1: bead coupling (Sec. 1: Stokes friction between beads and
 * fluid; reads the state, moves the chain, records the force density at
 * <= 8 sites per bead), fused stream-collide of all sites (D3Q19, Sec. 3)
 * with the boundary layer set to the equilibrium of the boundary velocity
 * at t = n+1 (Sec. 2; time interpolation of Sec. 3, after Eq. 1),
 * re-collision of the forced sites.
 *   Returns LB_ERR_STATE if a needed boundary sample has not been pushed.
 */
int32_t lb_step(lb_ctx* ctx, int32_t nsteps);

/*
 * lb_graph_capture / lb_graph_launch -- capture nsteps steps into a CUDA
 * graph owned by the context and replay it.  The graph reads the step
 * number from device memory, so each replay advances the state by nsteps.
 */
int32_t lb_graph_capture(lb_ctx* ctx, int32_t nsteps);
int32_t lb_graph_launch(lb_ctx* ctx);

/*
 * lb_read_fields -- observables of one box at the current step (Sec. 3: the
 * LB velocity field is what the paper compares with the DNS, Figs. 1-2).
 *   LB_FIELD_RHO / LB_FIELD_U: on boundary sites the moments of the stored
 *   equilibrium; elsewhere the moments of the pulled populations
 *   f_i(x) = A_i(x - c_i), u = (j + rho a / 2) / rho, a the body
 *   acceleration of the current step (body_accel plus, for a box with
 *   frame_accel, the frame acceleration at t_n).
 *   dst: host or device memory of the size given with the LB_FIELD_* code.
 *   Synchronising (bounded wait, see lb_sync); returns a pending box error.
 */
int32_t lb_read_fields(lb_ctx* ctx, int32_t box, int32_t what, void* dst);

/*
 * lb_conservation -- FP64 sums over all sites of a box:
 *   out[0] = sum_x sum_i f_i, out[1..3] = sum_x sum_i c_i f_i,
 *   out[4..6] = bead momentum m sum_b V_b.   out: host, 7 doubles.
 *   Synchronising; flags LB_ERR_NONFINITE for a non-finite sum.
 */
int32_t lb_conservation(lb_ctx* ctx, int32_t box, double* out);

/*
 * lb_vorticity -- mean magnitude of the vorticity over a cube of one box
 * (Sec. 3, Figs. 1 and 2: |omega| averaged over the whole sub-volume around
 * the tracer and over a small region at its centre, LB against DNS).
 *   u is the velocity lb_read_fields(LB_FIELD_U) reports; omega = curl u by
 *   second-order central differences, omega_x = (u_z(y+1) - u_z(y-1))/2 -
 *   (u_y(z+1) - u_y(z-1))/2 and cyclically, |omega| in FP64.
 *   lo, hi: the cube holds the sites with lo <= x, y, z <= hi; it must lie
 *   inside 1 .. E-2 (LB_ERR_ARG otherwise).
 *   out: host, one double: the mean of |omega| over the (hi - lo + 1)^3 sites.
 *   Uses the context's free population buffer as scratch (no allocation);
 *   the sum runs in a fixed order (the same inputs give the same result).
 *   Synchronising (bounded wait); returns a pending box error.
 */
int32_t lb_vorticity(lb_ctx* ctx, int32_t box, int32_t lo, int32_t hi, double* out);

/* lb_sync -- wait for the context stream at most timeout_ms (LB_ERR_TIMEOUT
 * after that, the context stays usable) and return the first box error.
 * The paper's replay runs about 1.85e5 LB steps per tracer (Sec. 3-4: one
 * DNS sample every 0.05 tau_eta over 81 tau_eta, about 113 LB steps per
 * sample by Eq. 1), so errors are collected at the caller's pace rather
 * than after every step. */
int32_t lb_sync(lb_ctx* ctx, int32_t timeout_ms);

/* lb_status -- device status word of a box (synchronising), LB_OK if clean. */

/*
 * lb_checkpoint_bytes / lb_save / lb_load -- checkpoint and restore of a
 * whole context, so that a long tracer replay (Sec. 3-4: about 1.85e5 LB
 * steps per tracer) can stop and resume exactly where it left off.
 *   A checkpoint holds the step counter and, for every box, its current
 *   populations, the boundary-ring slots, the frame-acceleration samples,
 *   the index of the last boundary sample pushed, its status word and its
 *   chain (description, bead positions and velocities); for upsampler boxes
 *   also the network output of the current coarse interval.  It does not
 *   hold the upsampler parameters: bind them again (lb_mlp_bind) after a
 *   load.  The launch settings (lb_set_launch, lb_set_bead_launch) are not
 *   part of the state.
 *   lb_checkpoint_bytes: size in bytes of a checkpoint of this context.
 *   lb_save: dst, host or device memory of that size.  Waits for every
 *   enqueued step (bounded wait), then copies; synchronising.
 *   lb_load: ctx must have been created with the same box descriptions,
 *   storage and ring_slots as the context saved (LB_ERR_ARG otherwise,
 *   nothing changed); src host or device.  Replaces the state of every box;
 *   the next lb_step continues from the saved step with the same result,
 *   bit for bit, as the run that was saved.  Drops a captured graph;
 *   synchronising.
 */
size_t lb_checkpoint_bytes(const lb_ctx* ctx);
int32_t lb_save(lb_ctx* ctx, void* dst);
int32_t lb_load(lb_ctx* ctx, const void* src);
int32_t lb_status(lb_ctx* ctx, int32_t box, int32_t* status);

/* lb_current_step -- number of steps enqueued so far. */
int64_t lb_current_step(const lb_ctx* ctx);

/* stream-collide kernels */
#define LB_KERNEL_STAGED 0    /* persistent, tiles staged in shared memory by TMA bulk copies, producer warp + 15 consumer warps */
#define LB_KERNEL_REGISTER 1  /* one vector load per population into registers, x-neighbours by warp shuffles */

/* lb_set_launch -- choice and launch shape of the stream-collide kernel.
 *   kernel LB_KERNEL_STAGED (default): 512 threads per block (one producer
 *   warp, 15 consumer warps), tiles of 480 x sites_per_thread sites staged
 *   in as many pipeline stages as fit in shared memory; threads must be 0;
 *   sites_per_thread 0 (default: 1 for FP64, 2 otherwise), 1, or 2 (not
 *   FP64); ctas = persistent grid (0 = one block per SM).
 *   kernel LB_KERNEL_REGISTER: threads per block (multiple of 32, 64 .. 256),
 *   ctas = persistent grid (0 = one block per tile), sites_per_thread
 *   (0 = default: 2 for FP64, 4 for FP32, 8 for 16-bit storage; half or a
 *   quarter of the default, at least 1, are the other choices).
 *   Used by the autotuner.  Drops a captured graph. */
int32_t lb_set_launch(lb_ctx* ctx, int32_t kernel, int32_t threads, int32_t ctas, int32_t sites_per_thread);

/* lb_set_bead_launch -- thread layout of the MD substeps of the bead
 *   kernel (Sec. 1: the chain dynamics of the hybrid method).
 *   lanes: threads per bead, 0 = default (the chain-order layout below), or
 *   1, 2, 4, 8; the lanes of a bead share its bond and pair
 *   forces and sum them by shuffles.  beads_per_thread: 1, or 2 with
 *   lanes = 1 (two beads per thread), or 0 with lanes = 2: the chain-order
 *   layout -- thread t holds bead t / 2; one lane of a bead takes its bonds,
 *   the other the beads two apart, the two split the Verlet list, every pair
 *   slot masked rather than branched.  One barrier over the MD threads per
 *   substep in every layout.  lanes x ceil(largest chain / beads_per_thread)
 *   <= 512.  Used by the autotuner; drops a captured graph.  LB_ERR_ARG
 *   otherwise. */
int32_t lb_set_bead_launch(lb_ctx* ctx, int32_t lanes, int32_t beads_per_thread);

/*
 * lb_set_chain_history -- the chain trajectory on the device (Sec. 1 and 4: the
 * method exists to follow a polymer chain's conformation in the flow).  After every
 * step n -> n + 1 the bead kernel writes the end-of-step positions of every
 * chain into slot (n + 1) mod slots of dev, so that a graph replay of several
 * steps leaves each step's positions to be read back at once.
 *   dev: device memory owned by the caller, 8-byte aligned, slots x 3 x
 *   (total bead capacity) doubles: chains in box order, each taking its
 *   box's bead capacity (nbeads of its description), bead b of a chain at
 *   its offset + b, x y z.  Valid until replaced or slots = 0.
 *   slots: ring length; 0 stops recording (dev ignored).
 *   A step whose box is flagged with an error writes nothing for that chain.
 *   Drops a captured graph.  LB_ERR_ARG for a negative slot count, a null
 *   or host buffer; LB_ERR_STATE when the context has no chain.
 */
int32_t lb_set_chain_history(lb_ctx* ctx, void* dev, int32_t slots);

/*
 * lb_set_fluctuation -- fluctuating collision for one box: the thermal fluid
 * of the hybrid method the paper builds on (Sec. 1, the Ahlrichs-Duenweg
 * coupling of a bead chain to a fluctuating lattice Boltzmann fluid).  The
 * collision acts on the 19 moments of the D3Q19 orthogonal basis e_k(c)
 * (sum_i w_i e_k(c_i) e_l(c_i) = b_k delta_kl; mass and momentum, k = 0..3,
 * conserved): m_k* = gamma_k m_k^neq + sqrt(mu rho b_k (1 - gamma_k^2)) xi_k
 * for k = 4..18 with mu = kT / c_s^2 = 3 kT, xi_k unit-variance uniforms from
 * Philox4x32-10 with counter (step, site, block 0..3, 0xF1) and key seed,
 * words 0..14 to modes 4..18; then f_i* = f_i^eq + w_i sum_k e_k(c_i) m_k* / b_k.
 * gamma_k = 1 - 1/tau for all k with kT = 0 is the BGK collision.
 *   gamma: host, 19 doubles (entries 0..3 ignored), each of 4..18 in (-1, 1);
 *   NULL switches the box back to BGK.  kT >= 0.
 *   Boundary sites of velocity faces keep their equilibrium.  Boxes with a
 *   chain capacity or a body force, and contexts on the register kernel, are
 *   refused (LB_ERR_ARG / LB_ERR_STATE): chains and forcing couple to BGK
 *   boxes only.  Drops a captured graph; synchronising.
 */
int32_t lb_set_fluctuation(lb_ctx* ctx, int32_t box, double kT, uint64_t seed, const double* gamma);

/*
 * lb_test_inject -- test only: make a device-side bounded wait run out, so
 * that the error path it guards can be exercised without faulting or hanging
 * the GPU (the paper has no counterpart; this serves the library's failure
 * detection).
 *   what = LB_INJECT_WITHHOLD_LAST_TILE: from the next stream-collide launch
 *   on, the producer of the staged kernel never arms the pipeline stage of
 *   the last tile of the tile list (the last box's last sites) and issues no
 *   copy for it.  The consumer warps waiting for that stage give up after
 *   the wait limit, set LB_ERR_TIMEOUT on the tile's box and leave; that box
 *   freezes, every other box steps on unaffected (the tiles a block took
 *   before the withheld one are finished first).  LB_INJECT_NONE turns the
 *   injection off.
 *   wait_limit_us: limit of the staged kernel's bounded barrier waits in
 *   microseconds, 1 .. 1000000 (0 = the default of one second).
 *   Needs the staged kernel (LB_ERR_STATE otherwise); lb_set_launch to the
 *   register kernel resets both settings.  Drops a captured graph.
 */
#define LB_INJECT_NONE 0
#define LB_INJECT_WITHHOLD_LAST_TILE 1
int32_t lb_test_inject(lb_ctx* ctx, int32_t what, int32_t wait_limit_us);

/*
 * lb_profile -- time every stream-collide launch with a pair of CUDA events
 * recorded on the context stream around it.  enable = 1 starts a new
 * measurement with room for max_launches launches (later launches are not
 * timed); enable = 0 stops recording.  lb_profile_read waits for the events
 * and returns the summed kernel time in milliseconds and the number of timed
 * launches.  Events are host-side objects; no device memory is used.
 */
int32_t lb_profile(lb_ctx* ctx, int32_t enable, int32_t max_launches);
int32_t lb_profile_read(lb_ctx* ctx, double* total_ms, int64_t* launches);

/* lb_last_error -- message of the last failing call on this context (or of
 * the last failing lb_plan / lb_create when ctx is NULL). */
const char* lb_last_error(const lb_ctx* ctx);

/*
 * Synthetic coarse flow (stands in for the paper's DNS sub-volume record,
 * Sec. 3: samples around a tracer every 0.05 tau_eta):
 *   u(x, t) = sum_m amp_m cos(kvec_m . (x - xc) + omega_m t + phi_m),
 *   xc = ((E-1)/2, (E-1)/2, (E-1)/2).
 * The mode table (kvec [M][3], amp [M][3], omega [M], phi [M], double,
 * M <= 3072) is in device memory.  Evaluated in FP64; out_dtype LB_STORE_F64
 * writes double, LB_STORE_F32 writes float.  workspace: device scratch of at
 * least lb_synth_workspace_bytes(M, E) bytes for the per-axis phase table.
 * Enqueued on `stream` (cudaStream_t); no synchronisation.
 *
 * Points: the coarse grid of a box with zoom z, 1 <= z <= E - 1 (see the
 * coarse-grid note above lb_box_desc; every site for z = 1).
 * lb_synth_faces: samples j0 .. j0+nsamp-1 at t = j K on the coarse points
 *   of the six face planes, out [nsamp][6][3][Ec][Ec] (device).
 * lb_synth_volume: the field at time t on the coarse grid, out [3][Ec^3]
 *   (device).
 */
size_t lb_synth_workspace_bytes(int32_t M, int32_t E);
int32_t lb_synth_faces(const double* kvec, const double* amp, const double* omega, const double* phi,
                       int32_t M, int32_t E, int32_t zoom, int32_t K, int64_t j0, int64_t nsamp, int32_t out_dtype,
                       void* out, void* workspace, void* stream);
int32_t lb_synth_volume(const double* kvec, const double* amp, const double* omega, const double* phi,
                        int32_t M, int32_t E, int32_t zoom, double t, int32_t out_dtype, void* out, void* workspace,
                        void* stream);

/*
 * Learned boundary upsampler (boxes with LB_TIME_MLP).  The paper
 * interpolates the DNS boundary linearly in time (Sec. 3); this added form
 * predicts, per face site and coarse interval j, the residual of the boundary
 * velocity over the cubic Hermite interpolant at the K substeps from the
 * samples j-1 (clamped to 0), j, j+1, j+2 and the in-face differences of
 * samples j and j+1 (24 features divided by u_max, zero-padded to 32).
 * Network 32 -> 128 -> 128 -> 3K with ReLU; bf16 weights and activations on
 * the tcgen05 tensor cores with TMEM accumulators (inference, and the forward
 * and backward of training; loss and Adam in FP32), f32 accumulation;
 * output row r = (f E + q) E + p holds
 * the residual of component c at substep s in units of u_max / 64 at
 * [3 (s-1) + c] (the residual is a few thousandths of u_max; a finer output
 * unit keeps the output weights at a scale Adam trains well).
 *
 * Inference parameters (device, lb_mlp_param_bytes(K) bytes, 256-byte
 * aligned sections): bf16 W1t [128][32], W2t [128][128], W3t [3K][128]
 * (output-major), then f32 b1 [128], b2 [128], b3 [3K].
 * Master parameters (f32, input-major like the CPU oracle): W1 [32][128],
 * b1 [128], W2 [128][128], b2 [128], W3 [128][3K], b3 [3K].
 *
 * lb_mlp_bind: boxes with LB_TIME_MLP use these parameters (borrowed until
 *   the context is destroyed or rebound); u_max scales features (1/u_max)
 *   and output (u_max/64).
 *   At every interval start lb_step first builds the features of those boxes
 *   from the ring and runs the network.
 * lb_mlp_features: feature matrix bf16 [6 E^2][32] of one face set from four
 *   samples [6][3][E][E] (real_dtype LB_STORE_F64 or LB_STORE_F32, device);
 *   X must be 16-byte aligned (LB_ERR_ARG otherwise).
 * lb_mlp_targets: training targets f32 [6 E^2][3K]: (fine - Hermite) * 64 / u_max
 *   with fine [K + 1][6][3][E][E] the boundary at t = jK .. jK + K;
 *   first_interval = 1 uses the one-sided tangent of interval 0.
 * lb_mlp_forward: Y f32 [rows][3K] from features X bf16 [rows][32].
 * Training (workspace of lb_mlp_train_bytes(K, batch_rows) bytes, device,
 * caller-owned): lb_mlp_train_init copies master parameters (host or device)
 * and clears the Adam moments; lb_mlp_grad runs forward and backward on
 * rows <= batch_rows of (X, T) and writes the f32 gradient in master layout
 * and the MSE loss (device pointers, either may be NULL); lb_mlp_train_step
 * does the same and applies one Adam step (lr, step t >= 1, betas 0.9 and
 * 0.999, eps 1e-8); lb_mlp_export writes the inference parameters.
 * All enqueue on `stream` without synchronising.
 */
size_t lb_mlp_param_bytes(int32_t K);
int32_t lb_mlp_bind(lb_ctx* ctx, const void* params, double u_max);
size_t lb_mlp_train_bytes(int32_t K, int64_t batch_rows);
int32_t lb_mlp_train_init(void* ws, int32_t K, int64_t batch_rows, const float* master, void* stream);
int32_t lb_mlp_features(const void* s_prev, const void* s0, const void* s1, const void* s2, int32_t real_dtype,
                        int32_t E, double u_max, void* X, void* stream);
int32_t lb_mlp_targets(const void* s_prev, const void* s0, const void* s1, const void* s2, const void* fine,
                       int32_t real_dtype, int32_t E, int32_t K, int32_t first_interval, double u_max, float* T,
                       void* stream);
int32_t lb_mlp_forward(const void* params, int32_t K, const void* X, int64_t rows, float* Y, void* stream);
int32_t lb_mlp_grad(void* ws, int32_t K, int64_t batch_rows, const void* X, const float* T, int64_t rows,
                    float* grad_out, double* loss_out, void* stream);
int32_t lb_mlp_train_step(void* ws, int32_t K, int64_t batch_rows, const void* X, const float* T, int64_t rows,
                          float lr, int64_t t, double* loss_out, void* stream);
int32_t lb_mlp_export(const void* ws, int32_t K, int64_t batch_rows, void* params, void* stream);

/*
 * lb_population_sums_noalloc -- FP64 sums of one box's population buffer,
 * for callers that cannot allocate device memory.  The paper has no
 * counterpart; this is a service of the library.
 *   Who needs it: a caller whose device memory is fully committed before the
 *   run (a framework caching allocator that has reserved the GPU, or a loop
 *   that forbids allocations after start-up to keep its footprint and
 *   latency fixed) cannot give lb_conservation a context arena.  This call
 *   needs only the populations and an output buffer.
 *   populations: device, [19][E][E][E] deviations f_i - w_i in `storage`
 *   format (LB_STORE_*), e.g. a LB_FIELD_DEV read-out.
 *   out: device, 4 doubles: sum_x sum_i f_i, then sum_x sum_i c_i f_i.
 *   stream: cudaStream_t the two kernels are enqueued on; no synchronisation.
 *   Scratch: a fixed array of 512 KiB compiled into the library (partial sums
 *   of at most 16384 blocks), held by every GPU that loads the library until
 *   the process exits.  No cudaMalloc, cudaFree or allocating library call.
 *   The first call on each device looks up the array's device address (one
 *   cudaGetSymbolAddress with that device current); make that first call
 *   before any stream capture.  The address is kept per device and CUDA
 *   context: after a device reset (cudaDeviceReset, or any new context on the
 *   device) the next call looks it up again, so the first-call rule applies
 *   again.  All calls share the array: calls that overlap on the GPU race; a
 *   call never reads a partial it has not written itself, so nothing needs
 *   clearing between calls.
 *   Errors: LB_ERR_SIZE if E > 400 (the array holds the partials of at most
 *   400^3 sites), LB_ERR_ARG for a null pointer, unknown storage or E < 1
 *   (both checked before any CUDA call), LB_ERR_CUDA if the address look-up
 *   or a launch fails; lb_last_error(NULL) gives the message.  The call has
 *   no size argument for the buffers: populations must hold 19 E^3 elements
 *   of the storage format and out 4 doubles, both device memory.
 */
int32_t lb_population_sums_noalloc(const void* populations, int32_t storage, int32_t E, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LBTRACER_H */
