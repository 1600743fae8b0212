/*
 * sim.h - C ABI of the GB300 batched articulated-body physics step.
 *
 * One physics step for thousands of independent environments resident on one GPU (Isaac Gym,
 * arXiv 2108.10470): reduced-coordinate articulations (Sec. "Physics Simulation"), ground contact
 * generation, a fixed-iteration TGS-style Gauss-Seidel contact and joint-limit solve (same
 * section, TGS paragraph and the simulation-parameter table), and integration. The state is
 * exposed as flat global tensors that the caller views without copying (Sec. "Tensor API";
 * tables "Physics state tensors" and "Physics control tensors").
 *
 * Conventions
 *   - Every call returns an int status: SIM_OK (0) or a negative SIM_ERR_* code; no call throws.
 *   - Model arrays passed to sim_create are HOST memory; they are validated and copied, and the
 *     caller keeps ownership.
 *   - The library owns every device buffer. Views (sim_get_view) alias them and stay valid until
 *     sim_destroy. All device work is enqueued on the stream given to sim_create (or
 *     sim_set_stream) and is asynchronous; reads of a view are valid in stream order.
 *   - Units: metres, kilograms, seconds, radians. World frame is z-up; the ground is the plane
 *     z = 0 with normal +z.
 *   - Quaternions are (x, y, z, w). Rotational inertia is (xx, yy, zz, xy, xz, yz) about the
 *     link's centre of mass, in link axes.
 */
#ifndef ARTSIM_SIM_H
#define ARTSIM_SIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------------- */
enum {
  SIM_OK = 0,
  SIM_ERR_INVALID_ARG = -1, /* null pointer, non-positive count, bad enum, non-finite number      */
  SIM_ERR_TOPOLOGY = -2,    /* parent[i] >= i, parent[0] != -1, root joint not FREE/FIXED, ...     */
  SIM_ERR_CUDA = -3,        /* a CUDA runtime call failed (message: sim_last_error_message)       */
  SIM_ERR_CAPACITY = -4,    /* an env exceeds the kernel limits (links, DOFs, shapes, candidates) */
  SIM_ERR_TIMEOUT = -5,     /* reserved: a bounded device wait gave up                            */
  SIM_ERR_NONFINITE = -6,   /* sim_sync_status: some env's state became NaN/Inf                    */
  SIM_ERR_HANDLE = -7,      /* null, destroyed or foreign handle                                   */
  SIM_ERR_NO_DEVICE = -8    /* no CUDA device is visible                                           */
};

/* ---- model description ----------------------------------------------------------------------- */
enum { SIM_JOINT_FREE = 0, SIM_JOINT_FIXED = 1, SIM_JOINT_REVOLUTE = 2, SIM_JOINT_PRISMATIC = 3,
       SIM_JOINT_SPHERICAL = 4 };
enum { SIM_SHAPE_SPHERE = 0, SIM_SHAPE_CAPSULE = 1, SIM_SHAPE_BOX = 2 };

/* One articulation (paper, Sec. "Physics Simulation": reduced-coordinate articulations; a single
 * rigid body is a one-link articulation). Links are numbered 0..n_links-1 with parent[i] < i and
 * parent[0] = -1; link 0 is the root and its joint_type is FREE (floating base, 6 DOF) or FIXED.
 * Every other link's joint is REVOLUTE or PRISMATIC (1 DOF about/along joint_axis, expressed in
 * the joint frame), SPHERICAL (a ball joint, 3 DOF: positions = the rotation vector r of the link
 * frame in the joint frame, R = exp([r]x), kept as the shorter rotation, |r| <= pi; velocities =
 * the link's angular velocity relative to its parent in link coordinates; RBDA Table 4.1; no
 * limits, drives or tendons; its env type runs a global-rows kernel variant) or FIXED. The joint frame of link i sits at
 * parent_pos[i] in the parent link's frame with orientation parent_quat[i]; at q = 0 the link
 * frame coincides with it. A multi-axis joint can also be a chain of 1-DOF joints through massless
 * "virtual" links (is_virtual = 1), which carry no shapes and are left out of the per-body tensors.
 * The DOF state rows of a joint follow link order, a ball joint's three in a row. Per-link joint data (armature = rotor
 * inertia added to the DOF, damping = viscous joint damping, limits) belong to the link's joint.
 * Shapes: SPHERE size[0] = radius; CAPSULE size[0] = radius, size[1] = half segment length, axis =
 * shape-local x; BOX size = half extents. A shape sits at shape_pos / shape_quat in its link's frame.
 * Array lengths: L = n_links, S = n_shapes; "[L*3]" means 3 floats per link, row-major. */
typedef struct {
  int32_t n_links;
  const int32_t* parent;      /* [L]                                                     */
  const int32_t* joint_type;  /* [L]   SIM_JOINT_*                                        */
  const float* joint_axis;    /* [L*3] unit axis in the joint frame (ignored if no DOF)   */
  const float* parent_pos;    /* [L*3]                                                     */
  const float* parent_quat;   /* [L*4] (x, y, z, w), normalised on copy                    */
  const float* mass;          /* [L]   >= 0; > 0 for a FREE root                           */
  const float* com;           /* [L*3] centre of mass in the link frame                    */
  const float* inertia;       /* [L*6] xx yy zz xy xz yz about the COM; positive semi-def. */
  const float* armature;      /* [L]   >= 0                                                */
  const float* damping;       /* [L]   >= 0                                                */
  const float* limit_lo;      /* [L]   used when has_limit[i]                              */
  const float* limit_hi;      /* [L]   >= limit_lo                                          */
  const uint8_t* has_limit;   /* [L]   0/1                                                  */
  const uint8_t* is_virtual;  /* [L]   0/1                                                  */
  int32_t n_shapes;
  const int32_t* shape_link;  /* [S]   link index, not virtual                              */
  const int32_t* shape_type;  /* [S]   SIM_SHAPE_*                                          */
  const float* shape_size;    /* [S*3] > 0 where used                                       */
  const float* shape_pos;     /* [S*3]                                                      */
  const float* shape_quat;    /* [S*4]                                                      */
  const float* shape_friction;/* [S]   >= 0                                                 */
  const float* drive_stiffness; /* [L] >= 0 joint drive stiffness kp, or NULL (no drives)   */
  const float* drive_damping;   /* [L] >= 0 joint drive damping kd, or NULL                  */
  int32_t n_tendons;            /* fixed tendons, 0..8 (0: the arrays below are ignored)      */
  const int32_t* tendon_joint_count; /* [T] 1..8 joints per tendon                             */
  const int32_t* tendon_link;   /* [sum counts] link of each joint (a 1-DOF joint), tendon by tendon */
  const float* tendon_coef;     /* [sum counts] length coefficient of each joint              */
  const float* tendon_stiffness;/* [T] >= 0                                                   */
  const float* tendon_damping;  /* [T] >= 0                                                   */
  const float* tendon_rest_length; /* [T]                                                     */
  const float* tendon_limit_lo; /* [T] used when tendon_has_limit                             */
  const float* tendon_limit_hi; /* [T] >= lo                                                  */
  const uint8_t* tendon_has_limit; /* [T] 0/1                                                 */
} sim_model_desc;
/* Fixed tendons (paper: fixed tendons coupling joints, with stiffness, damping and limits): the
 * length of a tendon is l = sum_k coef_k q_k over its joints; each substep it applies the force
 * -stiffness (l - rest) - damping l_dot (at the substep start) to each joint as coef_k times it,
 * and a limited tendon gets constraint rows (J = +-coef over its joints, treated like joint-limit
 * rows) when l is within the limit margin of lo or hi; lo = hi holds the length fixed. */
/* Joint drives (paper: DOF position / velocity targets with drive stiffness and damping): each
 * substep a driven joint gets the force kp (q* - q - h qd) + kd (qd* - qd) with h (h kp + kd)
 * added to its joint-space inertia diagonal, i.e. the spring-damper integrated implicitly over the
 * substep (stable for stiff gains); q*, qd* come from the DOF_POSITION_TARGET / _VELOCITY_TARGET
 * views. */

/* Solver parameters (paper's simulation-parameter table: gravity, position / velocity iteration
 * counts, max bias, friction; contact offset and limit margin are this library's constants).
 * flags: bit 0 (SIM_FLAG_SIGNATURE) records the per-env constraint-set signature each step;
 * bit 1 (SIM_FLAG_PERSISTENT) runs every env type of a step in one persistent launch instead of
 * one launch per env type; bit 2 (SIM_FLAG_GRAPH) makes sim_step capture its launches into a CUDA
 * graph on first use (again whenever dt or substeps change, or the plan changes) and replay it;
 * bit 3 (SIM_FLAG_BODY_FORCES) applies the RIGID_BODY_FORCE view every substep; bit 4
 * (SIM_FLAG_RIGID_BODY_STATE) writes the RIGID_BODY_STATE view after every step; bit 5
 * (SIM_FLAG_DOF_FORCE) writes the DOF_FORCE view every step; bit 6 (SIM_FLAG_ROW_SOLVER) runs
 * every substep's Gauss-Seidel solve in the row form (each row's J v and separation as group
 * reductions over Y = L^-1 J^T) instead of the Delassus form (W = J M^-1 J^T per substep, one
 * row value per lane), which is used otherwise whenever W fits beside Y; the two agree to FP32
 * rounding (paper, Sec. "Physics Simulation": the TGS solve; both forms keep its row order and
 * projections); bit 7 (SIM_FLAG_TANGENT_VJP) makes sim_step_vjp use the forward-mode derivative
 * kernel even where the reverse pass covers the step (a second, independent evaluation). */
enum { SIM_FLAG_SIGNATURE = 1, SIM_FLAG_PERSISTENT = 2, SIM_FLAG_GRAPH = 4, SIM_FLAG_BODY_FORCES = 8,
       SIM_FLAG_RIGID_BODY_STATE = 16, SIM_FLAG_DOF_FORCE = 32, SIM_FLAG_ROW_SOLVER = 64,
       SIM_FLAG_TANGENT_VJP = 128 };
typedef struct {
  float gravity[3];
  int32_t pos_iters;       /* >= 1 biased (position) iterations                  */
  int32_t vel_iters;       /* >= 0 unbiased (velocity) iterations                */
  float contact_offset;    /* a contact point is active iff separation < this    */
  float limit_margin;      /* a limit row is active iff distance to limit < this */
  float bias_coef;         /* fraction of the penetration corrected per iteration */
  float max_depen_vel;     /* cap on the push-out velocity                       */
  float ground_friction;   /* ground friction; a contact uses max(shape, ground) */
  int32_t flags;
} sim_params;

/* ---- views ----------------------------------------------------------------------------------- */
/* CONTACT_PAIRS rows: shape indices are env-local (actors in row order, shapes in model order);
 * shape_a is the shape on body a (the contact normal points from body b to body a). For a ground
 * contact slot is the sample on shape_a (sphere 0, capsule ends 0 and 1, box corners 0..7); for a
 * capsule-box pair it is 0 / 1 (capsule segment ends), 2 / 3 (ends of the segment part over the
 * box face or edge nearest the closest point) or 4 (closest point of segment and box). */
enum {
  SIM_VIEW_ROOT_STATE = 0,        /* (N_A, 13) f32 [p 3 | quat 4 | v 3 | omega 3] world; v = root origin velocity. Get/Set */
  SIM_VIEW_DOF_STATE = 1,         /* (N_D, 2)  f32 [q, qd]. Get/Set                                                        */
  SIM_VIEW_DOF_ACTUATION = 2,     /* (N_D,)    f32 joint force / torque applied during the next step. Set                   */
  SIM_VIEW_NET_CONTACT_FORCE = 3, /* (N_B, 3)  f32 net contact force on each (non-virtual) body, step average. Get          */
  SIM_VIEW_CONTACT_PAIRS = 4,     /* (n_envs, C, 3) i32 (shape_a, shape_b or -1 = ground, slot) of the step's last substep; padding -1 */
  SIM_VIEW_CONTACT_COUNT = 5,     /* (n_envs,) i32 number of valid rows in CONTACT_PAIRS                                     */
  SIM_VIEW_SIGNATURE = 6,         /* (n_envs,) u32 FNV-1a of the step's constraint sets (SIM_FLAG_SIGNATURE)                */
  SIM_VIEW_STATUS = 7,            /* (n_envs,) i32 per-env status bits: 1 non-finite state, 2 solver pivot failure           */
  SIM_VIEW_IMPULSE_CACHE = 8,     /* (n_envs, K) f32 warm-start impulses (solver state carried between substeps and steps)   */
  SIM_VIEW_DOF_POSITION_TARGET = 9,  /* (N_D,) f32 drive position targets q*. Set                                      */
  SIM_VIEW_DOF_VELOCITY_TARGET = 10, /* (N_D,) f32 drive velocity targets qd*. Set                                     */
  SIM_VIEW_DOF_FORCE = 11,        /* (N_D,) f32 joint force of the last substep: actuation - damping qd + drive (SIM_FLAG_DOF_FORCE). Get */
  SIM_VIEW_RIGID_BODY_STATE = 12, /* (N_B, 13) f32 per body after the step: link origin 3 | quat xyzw (w >= 0) 4 | origin velocity 3 | omega 3, world (SIM_FLAG_RIGID_BODY_STATE). Get */
  SIM_VIEW_RIGID_BODY_FORCE = 13  /* (N_B, 6) f32 per body: force 3 | torque 3, world axes, applied at the body's COM every substep (SIM_FLAG_BODY_FORCES). Set */
};
enum { SIM_DTYPE_F32 = 0, SIM_DTYPE_I32 = 1, SIM_DTYPE_U32 = 2 };
typedef struct {
  void* data;          /* device pointer owned by the library */
  int32_t ndim;
  int64_t shape[3];
  int64_t strides[3];  /* in elements */
  int32_t dtype;       /* SIM_DTYPE_* */
  int32_t device;      /* CUDA device ordinal */
} sim_view;

typedef struct sim_s* sim_handle;

/* Create a simulation of n_envs environments. Row e of env_actor_model (host array, n_envs x
 * actors_per_env, actors_per_env <= 8) lists the model indices of env e's actors; entries of -1
 * pad envs with fewer actors (every env needs at least one). Actor roots are numbered env-major,
 * then in row order, in the root tensor (N_A = number of non-negative entries); joint DOFs and
 * non-virtual bodies are numbered env-major, then actor, then link. Envs with the same actor list
 * form one env type (one launch per type and step). Within an env, shapes of different actors
 * collide pairwise when one is a capsule and the other a box; every shape collides with the
 * ground plane z = 0. cuda_stream is a cudaStream_t (NULL = legacy default stream). Initial
 * state: every root at its origin with identity orientation, zero velocities and joint
 * positions, zero actuation. Errors: INVALID_ARG, TOPOLOGY, CAPACITY (more than 32 links, 32
 * generalized DOFs, 32 shapes, 32 capsule-box pairs or 256 contact candidates in one env), CUDA,
 * NO_DEVICE; *out is set only on success. Environments never interact (paper: each environment
 * is simulated without interaction with the others). */
int sim_create(const sim_model_desc* models, int32_t n_models, const int32_t* env_actor_model,
               int32_t actors_per_env, int32_t n_envs, const sim_params* params, void* cuda_stream,
               sim_handle* out);

/* Advance every environment by dt using `substeps` equal substeps (paper: control dt vs.
 * simulation dt). Each substep: forward kinematics, articulated-body forward dynamics, ground and
 * capsule-box contact rows and joint-limit rows, pos_iters + vel_iters TGS-style Gauss-Seidel iterations,
 * integration. Reads DOF_ACTUATION, updates ROOT_STATE, DOF_STATE, NET_CONTACT_FORCE, the contact
 * views, IMPULSE_CACHE and STATUS. Asynchronous on the handle's stream. Errors: HANDLE,
 * INVALID_ARG (dt <= 0 or non-finite, substeps < 1), CUDA (launch failure). */
int sim_step(sim_handle h, float dt, int32_t substeps);

/* The step with this step's DOF actuation forces given by the caller (paper: applying an actuation
 * force tensor, set_dof_actuation_force_tensor, then simulate): `actuation` holds N_D floats in the
 * DOF_ACTUATION layout, in memory the device can read (device memory of the handle's device,
 * managed memory, pinned host memory) or any other host memory. On a handle of one env type the
 * step kernel loads the forces straight from a buffer the device can address and stores them into
 * DOF_ACTUATION, so no copy is launched; other buffers, and every buffer of a handle with several
 * env types or with SIM_FLAG_GRAPH or SIM_FLAG_PERSISTENT, are copied into DOF_ACTUATION on the
 * handle's stream first. Either way the views end exactly as after
 * writing DOF_ACTUATION and calling sim_step. The buffer is read asynchronously on the handle's
 * stream and must not change until the step has run; the caller keeps its ownership. Errors as
 * sim_step; INVALID_ARG for a NULL buffer when the handle has DOFs. */
int sim_step_actuated(sim_handle h, const float* actuation, float dt, int32_t substeps);

/* End-to-end step from host memory: host_actuation (N_D floats) into DOF_ACTUATION, sim_step,
 * ROOT_STATE (N_A*13 floats) and DOF_STATE (N_D*2 floats) into the host buffers (either output may
 * be NULL), then a stream synchronisation. Pinned buffers (CUDA-allocated or registered host
 * memory, which the device addresses) are read and written by the step kernels themselves: no
 * copy is launched; pageable buffers, and every buffer of a SIM_FLAG_GRAPH or SIM_FLAG_PERSISTENT
 * handle, are copied.
 * Either way the views end as after sim_step. Errors as sim_step. */
int sim_step_host(sim_handle h, const float* host_actuation, float* host_root_out, float* host_dof_out,
                  float dt, int32_t substeps);

/* ---- step without allocation ------------------------------------------------------------------
 * The paper has no counterpart to this call; it serves callers that cannot allocate device
 * memory when they step: a host application that hands out all device memory from a pool it
 * reserved up front, or a control loop that must not enter the driver's allocator while it runs.
 * They create the handle once, at set-up, and then step on state buffers they own.
 *
 * Caller-owned state, one device pointer per view of the same name, with that view's shape and
 * element layout (sizes from sim_get_sizes; C = contact pairs per env, K = impulse-cache length
 * per env). The library never frees or keeps these pointers beyond the call. */
typedef struct {
  float* root_state;          /* (N_A, 13) read and written */
  float* dof_state;           /* (N_D, 2) read and written (any 4-byte-aligned buffer when N_D = 0) */
  const float* dof_actuation; /* (N_D,) read */
  float* net_contact_force;   /* (N_B, 3) written */
  float* impulse_cache;       /* (n_envs, K) read and written; zero it for a fresh start */
  int32_t* contact_pairs;     /* (n_envs, C, 3) written */
  int32_t* contact_count;     /* (n_envs,) written */
  uint32_t* signature;        /* (n_envs,) written when SIM_FLAG_SIGNATURE is set */
  int32_t* status;            /* (n_envs,) written */
} sim_state_buffers;

/* The step of sim_step on the buffers in *io, with no device allocation in the call: env types
 * whose contact and row blocks do not fit in shared memory keep them in a scratch array built
 * into the library (64 MiB, a file-scope device array: every device where the library's device
 * code is loaded holds it until the process exits) instead of the handle's own scratch. The
 * handle supplies only the model tables, its launch plan and its stream; its views are neither
 * read nor written. Steps that would use them are refused with INVALID_ARG: handles created with
 * SIM_FLAG_BODY_FORCES (reads the RIGID_BODY_FORCE view), SIM_FLAG_RIGID_BODY_STATE or
 * SIM_FLAG_DOF_FORCE (write those views), and env types with joint drives (read the target views).
 * Handles with SIM_FLAG_PERSISTENT or SIM_FLAG_GRAPH step here with one launch per env type on
 * the handle's stream, without a graph.
 * Limit: each such env type needs its env count, rounded up to a whole CTA (128 / G envs, G the
 * lanes per env), times its per-env scratch within 64 MiB (a hand-with-cube env uses about 62 KB,
 * so about 1050 of them fit); a larger type fails with CAPACITY and a message giving the sizes,
 * before anything is launched. Env types that fit in shared memory have no limit: they step with
 * their whole row capacity in shared memory (sim_step may hold part of it in global slots of the
 * handle), which fails with CAPACITY only for a type whose knobs were set so that its CTA's arena
 * exceeds 220 KB.
 * Address: each call outside a stream capture looks up the array's device address on the
 * handle's device (with that device made current, the caller's device restored), so a device
 * reset between calls is followed; a call during a capture reuses the address of the last call on
 * that device, so make a first call before any stream capture (one made during a capture fails
 * with INVALID_ARG).
 * Sharing: every call, from every handle on a device, uses the same array, which keeps the last
 * call's contents. Nothing in it needs to start at zero (each step writes every scratch word
 * before reading it). Calls whose kernels overlap on the GPU (different streams without ordering
 * between them) race on the array and give wrong results: order them on one stream or with
 * events. Asynchronous on the handle's stream. Errors: HANDLE, INVALID_ARG (a NULL buffer,
 * dt <= 0 or non-finite, substeps < 1, the refused flags and drives above, a first call during a
 * capture), CAPACITY (above), CUDA. */
int sim_step_static_scratch(sim_handle h, const sim_state_buffers* io, float dt, int32_t substeps);

/* ---- launch plan --------------------------------------------------------------------------------
 * Envs with the same actor list form an env type. Each type is stepped with a kernel variant
 * chosen by three knobs: lanes per env (8, 16 or 32; at least the type's largest count of links,
 * generalized DOFs or shapes), where the solver's contact and row blocks live (shared memory, or
 * a per-env slot of global scratch; types with capsule-box pairs always use global scratch), and
 * warps per CTA of its per-type launch (1, 2 or 4). sim_create picks the fewest lanes, shared
 * rows when the env's arena is at most 24 KB, and 4 warps. (Paper: thousands of environments of
 * possibly different articulations packed into one simulation; the tuning is this library's.) */

/* Knobs of env type `type` (0 .. out[5] of sim_get_sizes - 1, in order of first appearance):
 * out[0] lanes per env, out[1] 1 if rows are in global scratch, out[2] warps per CTA, out[3]
 * number of envs of the type, out[4] fewest lanes the type allows, out[5] lowest env index of the
 * type. Errors: HANDLE, INVALID_ARG. */
int sim_get_type_config(sim_handle h, int32_t type, int32_t* out);

/* Set the knobs of env type `type`; results do not depend on them beyond FP32 rounding of
 * reductions. Synchronises the device when scratch must grow. Drops a captured graph. Errors:
 * HANDLE, INVALID_ARG (knob out of range, lanes below the type's minimum, shared rows for a type
 * with shape pairs), CAPACITY (the CTA's arena exceeds 220 KB, or a persistent launch no longer
 * fits), CUDA. */
int sim_set_type_config(sim_handle h, int32_t type, int32_t lanes_per_env, int32_t rows_global,
                        int32_t warps_per_cta);

/* Autotuner: time candidate knobs on the handle's current state and keep the fastest. Without
 * SIM_FLAG_PERSISTENT each type is tuned on its own launch over every valid (lanes, rows, warps);
 * with it, (lanes, rows) of each type in turn are tried on the whole persistent step (two passes
 * of coordinate descent). Each candidate is timed with CUDA events over `reps` steps (1..1000)
 * after one warm-up step, each step starting from a snapshot of every state tensor, and replaces
 * the knobs held so far (first the handle's current ones) only when its median step is at least
 * 3 % faster; the snapshot
 * is restored at the end, so the visible state is unchanged. *ms_per_step receives the chosen
 * plan's median step time. Synchronises the stream; allocates the snapshot for the call's
 * duration. Errors: HANDLE, INVALID_ARG, CUDA. */
int sim_autotune(sim_handle h, float dt, int32_t substeps, int32_t reps, double* ms_per_step);

/* ---- derivative of the step ---------------------------------------------------------------------
 * The env-step is differentiated with its constraint set and active set held fixed (contact and
 * limit decisions, clamps and the choice of solver target follow the values, as in the forward
 * step). The state that carries into the next step is (root state, DOF state, impulse cache); the
 * actuation is the step's control input. Net contact forces and the contact views are not
 * differentiated. Joint drives act as in the step, with the handle's DOF_POSITION_TARGET /
 * DOF_VELOCITY_TARGET views as constants (no gradient with respect to the targets), and so do the
 * RIGID_BODY_FORCE view's forces under SIM_FLAG_BODY_FORCES; tendon springs and tendon-limit rows
 * are differentiated, and so are capsule-box pair contacts.
 * Two evaluations. The reverse pass (sim_step_taped + sim_step_adjoint below) covers every env
 * type (shape pairs, ball joints, tendons, drives and SIM_FLAG_BODY_FORCES included); there the
 * gradient w.r.t. a root quaternion is its component tangent to the unit sphere (the step's
 * dependence on |q| is an artefact of the formulation: the output quaternion is normalised).
 * Otherwise (and under SIM_FLAG_TANGENT_VJP) forward-mode dual arithmetic, one env per warp, each
 * lane carrying up to 8 input directions, in passes of 256 directions per env, for env types whose
 * impulse cache has at most 448 entries (other handles fail with CAPACITY).
 * (The paper does not differentiate its step; this is the project's own extension, following the
 * paper's remark that its operational-space controller is differentiable, Sec. "Franka cube
 * stacking".) */
typedef struct {
  const float* root_state;           /* (N_A, 13) state at the start of the step */
  const float* dof_state;            /* (N_D, 2) */
  const float* dof_actuation;        /* (N_D,) */
  const float* impulse_cache;        /* (n_envs, K) */
  const float* grad_root_state;      /* (N_A, 13) gradient w.r.t. the step's output root state; NULL = 0 */
  const float* grad_dof_state;       /* (N_D, 2) w.r.t. the output DOF state; NULL = 0 */
  const float* grad_impulse_cache;   /* (n_envs, K) w.r.t. the output impulse cache; NULL = 0 */
  float* grad_root_state_in;         /* (N_A, 13) out: gradient w.r.t. root_state */
  float* grad_dof_state_in;          /* (N_D, 2) out */
  float* grad_dof_actuation;         /* (N_D,) out */
  float* grad_impulse_cache_in;      /* (n_envs, K) out (zero past each env type's cache length) */
  int32_t* status;                   /* (n_envs,) out, optional: 0, or 2 if the env's step failed
                                      * (pivot, or more than 64 contacts); its gradient is then 0 */
} sim_vjp_buffers;

/* Vector-Jacobian product of one env-step (substeps of dt / substeps) at the given input state:
 * every output gradient entry is contracted with the step's Jacobian. All pointers are device
 * memory owned by the caller, in the layouts of the views of the same names; the handle supplies
 * the model and its stream, its views are not touched (the reverse pass steps a library-owned copy
 * of the input state, allocated on first use). Asynchronous. Errors: HANDLE, INVALID_ARG (a
 * required pointer NULL: the DOF-state and actuation buffers may be NULL when the handle has no
 * joint DOFs; dt or substeps invalid), CAPACITY (unsupported env type), CUDA. */
int sim_step_vjp(sim_handle h, const sim_vjp_buffers* b, float dt, int32_t substeps);

/* ---- reverse pass of a recorded step ------------------------------------------------------------
 * The rollout pattern of a differentiable simulation: step forward recording each step's tape,
 * then apply the steps' adjoints in reverse order. The tape of one step holds, per env and
 * substep, the substep's input state, its contact and constraint-row lists, the joint-space
 * factor L and Y = L^-1 J^T, the generalized acceleration, the solve's vectors and each row
 * update's impulse and separation (and, for a capsule-box pair contact, its second body, normal
 * and the two actors' offset); everything else is recomputed by the adjoint. Covered: every env
 * type whose adjoint arena fits a CTA (otherwise CAPACITY; sim_step_vjp then differentiates in
 * forward mode). */

/* Floats of one step's tape (caller-owned device memory: allocate this many floats per recorded
 * step; the size depends on the handle's env types, solver iterations and substeps). Errors:
 * HANDLE, INVALID_ARG (substeps < 1, or the handle is not covered), CAPACITY. */
int sim_tape_size(sim_handle h, int32_t substeps, int64_t* floats);

/* One step of the handle's own state, exactly as sim_step computes it (the same kernel code and
 * arithmetic, one launch per env type whatever the handle's launch plan), that also writes the
 * step's tape to `tape` (device, sim_tape_size floats). The tape stays valid until it is
 * overwritten; it does not refer to the handle's views. Asynchronous. Errors: HANDLE, INVALID_ARG,
 * CAPACITY, CUDA. */
int sim_step_taped(sim_handle h, float* tape, float dt, int32_t substeps);

typedef struct {
  const float* grad_root_state;      /* (N_A, 13) gradient w.r.t. the step's output root state; NULL = 0 */
  const float* grad_dof_state;       /* (N_D, 2) w.r.t. the output DOF state; NULL = 0 */
  const float* grad_impulse_cache;   /* (n_envs, K) w.r.t. the output impulse cache; NULL = 0 */
  float* grad_root_state_in;         /* (N_A, 13) out: gradient w.r.t. the step's input root state */
  float* grad_dof_state_in;          /* (N_D, 2) out */
  float* grad_dof_actuation;         /* (N_D,) out */
  float* grad_impulse_cache_in;      /* (n_envs, K) out (zero past each env's read slots) */
  int32_t* status;                   /* (n_envs,) out, optional: 0, or 2 if a gradient is not finite */
} sim_adjoint_buffers;

/* Vector-Jacobian product of the step recorded in `tape` by sim_step_taped (same dt and substeps):
 * the output gradients in, the input gradients out (device memory owned by the caller, in the
 * layouts of the views of the same names; outputs may alias nothing else). One launch per env
 * type, one env per group of lanes, substeps in reverse order; the step's constraint and active
 * sets are those recorded (the DOF gradient buffers may be NULL when the handle has no joint
 * DOFs). Asynchronous. Errors: HANDLE, INVALID_ARG, CAPACITY, CUDA. */
int sim_step_adjoint(sim_handle h, const float* tape, const sim_adjoint_buffers* b, float dt, int32_t substeps);

typedef struct {
  const float* root_state;           /* (N_A, 13) state at the start of the step */
  const float* dof_state;            /* (N_D, 2) */
  const float* dof_actuation;        /* (N_D,) */
  const float* impulse_cache;        /* (n_envs, K) */
  const float* tan_root_state;       /* (N_A, 13) input tangent */
  const float* tan_dof_state;        /* (N_D, 2) */
  const float* tan_dof_actuation;    /* (N_D,) */
  const float* tan_impulse_cache;    /* (n_envs, K) */
  float* root_state_out;             /* (N_A, 13) out: the step's output, evaluated by the same serial code */
  float* dof_state_out;              /* (N_D, 2) out */
  float* impulse_cache_out;          /* (n_envs, K) out */
  float* tan_root_state_out;         /* (N_A, 13) out: output tangent */
  float* tan_dof_state_out;          /* (N_D, 2) out */
  float* tan_impulse_cache_out;      /* (n_envs, K) out */
  int32_t* status;                   /* (n_envs,) out, optional, as in sim_vjp_buffers */
} sim_jvp_buffers;

/* Jacobian-vector product of one env-step: the output state and its tangent along the given input
 * tangent. Same conventions and errors as sim_step_vjp. */
int sim_step_jvp(sim_handle h, const sim_jvp_buffers* b, float dt, int32_t substeps);

/* Largest generalized-DOF count (n_max) and link count (L_max) over the env types (the padded
 * sizes of the mass-matrix and Jacobian outputs). Errors: HANDLE, INVALID_ARG. */
int sim_get_max_dims(sim_handle h, int32_t* n_max, int32_t* l_max);

/* Joint-space inertia of every env at the current state (paper: mass matrices per actor group):
 * out (device, n_envs x n_max x n_max f32, row-major per env; entries past the env's generalized
 * DOFs are 0) receives M, armature included, for the generalized velocity [omega; p_dot] of each
 * floating root (world axes) followed by the joint rates, actors in order. Asynchronous on the
 * handle's stream. Errors: HANDLE, INVALID_ARG, CUDA. */
int sim_compute_mass_matrix(sim_handle h, float* out);

/* World-axis Jacobians of every link of every env at the current state (paper: Jacobian tensors):
 * out (device, n_envs x L_max x 6 x n_max f32) row r of link l maps the env's generalized velocity
 * to [angular velocity; velocity of the link origin] (rows past 6, links past the env's, columns
 * past its DOFs are 0). Asynchronous. Errors: HANDLE, INVALID_ARG, CUDA. */
int sim_compute_jacobian(sim_handle h, float* out);

/* Describe one of the SIM_VIEW_* device tensors. Errors: HANDLE, INVALID_ARG. */
int sim_get_view(sim_handle h, int32_t which, sim_view* out);

/* Apply new root states to an indexed subset of actors (paper, Sec. "Physics State Tensors":
 * set root or DOF states for all actors or a subset given by an index buffer). dev_src is a device
 * array (n, 13) of root rows, dev_actor_idx a device array of n global actor indices (out-of-range
 * indices are ignored). Teleports the roots without changing joint states, and clears the solver
 * impulse cache of the touched environments. Errors: HANDLE, INVALID_ARG (n < 0), CUDA. */
int sim_set_root_state_indexed(sim_handle h, const float* dev_src, const int32_t* dev_actor_idx, int32_t n);

/* Apply new DOF states to an indexed subset of environments: dev_src is a device array of n rows,
 * each holding one environment's joint DOF states (env_jdof x 2 floats, the env's own count;
 * all envs of a batch with mixed sizes use the largest count as row stride), dev_env_idx a device
 * array of n env indices (out-of-range ignored). Leaves root states unchanged and clears the
 * touched environments' impulse caches. Errors: HANDLE, INVALID_ARG, CUDA. */
int sim_set_dof_state_indexed(sim_handle h, const float* dev_src, const int32_t* dev_env_idx, int32_t n);

/* Replace the stream used by later calls. Errors: HANDLE. */
int sim_set_stream(sim_handle h, void* cuda_stream);

/* Synchronise the stream and count envs whose status word is non-zero. Returns SIM_OK when all
 * are clean, SIM_ERR_NONFINITE otherwise (*n_bad_envs receives the count). */
int sim_sync_status(sim_handle h, int32_t* n_bad_envs);

/* Sizes: out[0] = N_A, out[1] = N_D, out[2] = N_B, out[3] = contact pairs per env (C),
 * out[4] = impulse-cache floats per env (K), out[5] = number of env types, out[6] = kernel
 * launches per sim_step. Errors: HANDLE, INVALID_ARG. */
int sim_get_sizes(sim_handle h, int64_t* out);

/* Release every device buffer; the handle becomes invalid. Errors: HANDLE. */
int sim_destroy(sim_handle h);

/* Static string for a status code. */
const char* sim_error_string(int code);

/* Text of the last CUDA error seen by any call of this thread (empty if none). */
const char* sim_last_error_message(void);

/* FP32 FMA throughput probe (measurement of the CUDA-core roofline, which the step is bound by):
 * runs a dependent-chain-free FMA loop on every SM for `iters` iterations and returns the achieved
 * FP32 FLOP/s (2 per FMA) in *flops_per_s. Synchronous. Errors: INVALID_ARG, CUDA. */
int sim_probe_fp32_peak(void* cuda_stream, int32_t iters, double* flops_per_s);

#ifdef __cplusplus
}
#endif
#endif /* ARTSIM_SIM_H */
