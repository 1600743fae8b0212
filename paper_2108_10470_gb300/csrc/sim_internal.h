// Internal data layout of the GB300 articulated-body step: per-env-type model tables, the
// per-environment shared-memory arena, and the step kernel's argument block. Shared by the
// host-side C ABI (sim_api.cu) and the kernels (step_kernel.cuh); not part of the public ABI.
#pragma once
#include <cstdint>

namespace artsim {

// Kernel limits (one environment is handled by one group of G <= 32 lanes: a lane per link, per
// generalized DOF, per shape).
constexpr int kMaxLinks = 32;   // links per environment (all actors)
constexpr int kMaxGen = 32;     // generalized DOFs per environment (6 per floating root + joints)
constexpr int kMaxShapes = 32;  // shapes per environment
constexpr int kMaxPairs = 32;   // capsule-box shape pairs per environment
constexpr int kPairSlots = 5;   // samples per pair: t = 0, t = 1, face-clip entry / exit, closest point
constexpr int kMaxCand = 256;   // contact candidate points per environment
constexpr int kMaxActors = 8;   // actors per environment
constexpr int kMaxTendons = 8;      // fixed tendons per environment
constexpr int kMaxTendonJoints = 8; // joints per tendon

enum JointType : int { kFree = 0, kFixed = 1, kRevolute = 2, kPrismatic = 3, kSpherical = 4 };
enum ShapeType : int { kSphere = 0, kCapsule = 1, kBox = 2 };
enum RowKind : int { kRowLimit = 0, kRowNormal = 1, kRowFriction = 2, kRowTendon = 3 };

// One environment type = one sequence of actor models, flattened into a forest of links.
// Per-link arrays are indexed by the env-local link number (actors in order, links in order, so
// parents precede children and generalized DOFs increase along every root-to-leaf path).
struct EnvTypeTable {
  int n_links, n_gen, n_jdof, n_shapes, n_cand, n_body, n_actors, max_depth;
  int lim_cap, row_cap, cache_len, group;  // group = lanes per environment (8, 16 or 32)
  // per link
  int parent[kMaxLinks];        // env-local parent, -1 for an actor root
  int jtype[kMaxLinks];
  int depth[kMaxLinks];         // 0 for actor roots
  int first_child[kMaxLinks];   // children in ascending order: first_child, next_sibling chain
  int next_sibling[kMaxLinks];
  int gdof[kMaxLinks];          // first generalized DOF of the link's joint (-1: none)
  int jdof[kMaxLinks];          // first env joint-DOF index (DOF state row within the env) or -1
  int body[kMaxLinks];          // env body index (net-contact-force row) or -1 (virtual)
  int actor[kMaxLinks];
  int aroot[kMaxLinks];         // link index of the actor's root
  unsigned anc[kMaxLinks];      // bit g set iff generalized DOF g belongs to an ancestor-or-self
  int lim_slots[kMaxLinks];     // number of limit rows this joint can produce (0, 1 or 2)
  float axis[3][kMaxLinks];     // joint axis in the joint frame
  float ppos[3][kMaxLinks];     // joint frame origin in the parent frame
  float prot[9][kMaxLinks];     // joint frame rotation (row-major, joint -> parent)
  float mass[kMaxLinks];
  float com[3][kMaxLinks];
  float inertia[6][kMaxLinks];  // xx yy zz xy xz yz about the COM, link axes
  float armature[kMaxLinks], damping[kMaxLinks], lo[kMaxLinks], hi[kMaxLinks];
  int has_limit[kMaxLinks];
  float drive_kp[kMaxLinks], drive_kd[kMaxLinks];  // joint drive gains (0: no drive)
  int has_drives;
  int has_ball;  // the type has ball joints (3 DOF; global-rows variant only)
  // fixed tendons (env-local links of 1-DOF joints); limit rows follow the joint-limit rows and use
  // impulse-cache slots 3 n_cand + 2 n_jdof + 2 t + side
  int n_tendons;
  int ten_n[kMaxTendons];
  int ten_link[kMaxTendons][kMaxTendonJoints];
  float ten_coef[kMaxTendons][kMaxTendonJoints];
  float ten_k[kMaxTendons], ten_d[kMaxTendons], ten_rest[kMaxTendons], ten_lo[kMaxTendons], ten_hi[kMaxTendons];
  int ten_has_limit[kMaxTendons];
  // per shape
  int shape_link[kMaxShapes], shape_type[kMaxShapes], cand_off[kMaxShapes];
  float shape_size[3][kMaxShapes], shape_pos[3][kMaxShapes], shape_rot[9][kMaxShapes];
  float shape_mu[kMaxShapes];   // max(shape friction, ground friction)
  float shape_fr[kMaxShapes];   // the shape's own friction (pairs use max over the two shapes)
  // capsule-box pairs (env-local shape indices a < b, different actors), candidates after the
  // ground candidates: n_ground_cand + kPairSlots * pair + slot
  int n_pairs, n_ground_cand;
  int pair_a[kMaxPairs], pair_b[kMaxPairs];
  // per generalized DOF
  int dof_link[kMaxGen];
  int dof_comp[kMaxGen];        // 0..5 for a floating root ([omega; v]), -1 for a joint DOF
};

// Per-environment arena (offsets in 4-byte words). The link hand-off slots of the inward sweep
// (phase 1) and the constraint response Y (phase 2) alias. When an env type's worst case does not
// fit in shared memory ("global rows"), the contact and row blocks (con, Y, rowc, lam, rowa) live
// in a private per-env slot of global scratch memory instead (offsets relative to the slot), and
// the link slots get a shared-memory region of their own.
struct SmemLayout {
  int grows;  // 1: contact and row blocks in global scratch
  int scratch_words;  // words per group slot of global scratch: the contact and row blocks (grows), or
                      // Y for the substeps whose rows exceed ywords (a compact shared-rows layout); 0: none
  int link;   // kLinkWords per link: IA 21 | pA 6 | Ic 10
  int Y;      // n_gen x RS: Y = L^-1 J^T, one column per constraint row
  int RS;     // row stride of Y (odd)
  int SD;     // 6 per generalized DOF: motion subspace in world axes about the actor origin
  int M;      // n_gen x MS (MS odd): Cholesky factor L of the joint-space inertia (lower)
  int MS;
  int vec;    // 5 x n_gen: qdd | v0 | vf | dq | Linv
  int con;    // kConWords x ccap (SoA)
  int ccap;
  int rowc;   // float4 x rcap: row headers (16-byte aligned)
  int lam;    // rcap: impulses
  int rowa;   // rcap: row aux (DOF / contact index)
  int rcap;
  int frc;    // 3 per link
  int ball;   // kBallWords per link: ball-joint state and sweep blocks, global rows only
  int ywords; // words from Y to the end of its region: Y (n_gen x (R | 1) for R rows), then the
              // solver's Delassus block R x R and R accumulated impulses when they fit
  int total;  // words per environment (multiple of 4; = G mod 32 when groups share a warp)
};
constexpr int kLinkWords = 37;
constexpr int kBallWords = 36;  // per ball-joint link: U 18 | D^-1 6 | u 3 | q 3 | qd 3 | tau 3
// contact record (SoA): x y z (relative to actor a's origin) | d | mu | link_a | cand | shape_a |
// slot | link_b (-1: ground) | shape_b | n x y z (from b to a) | O_b - O_a x y z
constexpr int kConWords = 17;

// Arguments shared by every env type of a step.
struct StepArgs {
  // global tensors
  float* root;               // (N_A, 13)
  float* dof;                // (N_D, 2)
  const float* act;          // (N_D,) (device memory, or pinned host memory the device addresses)
  float* act_copy;           // non-null: every actuation value read is also stored here (the view)
  float* root_out;           // non-null: the step's final root rows are also stored here
  float* dof_out;            // non-null: the step's final DOF rows are also stored here
  float* net_force;          // (N_B, 3)
  float* cache;              // (n_envs, cache_stride)
  int* pairs;                // (n_envs, pair_stride, 3)
  int* n_pairs;              // (n_envs,)
  unsigned* sig;             // (n_envs,)
  int* status;               // (n_envs,)
  const int* env_dof_base;   // (n_envs,) first DOF row
  const int* env_body_base;  // (n_envs,) first body row
  const int* env_actor_base; // (n_envs,) first root-state row
  const float* pos_target;   // (N_D,) drive targets (read when the type has drives)
  const float* vel_target;   // (N_D,)
  const float* body_force;   // (N_B, 6) external force, torque (flag 8)
  float* dof_force;          // (N_D,) out (flag 32)
  float* body_state;         // (N_B, 13) out (flag 16)
  int cache_stride, pair_stride;
  // step
  float dt, h;
  int substeps;
  // parameters
  float gx, gy, gz;
  int pos_iters, vel_iters;
  float contact_offset, limit_margin, bias_coef, max_depen_vel;
  int flags;
};

// Tape of one env-substep, written by the taped instantiation of the step kernel for the reverse
// pass (offsets in 4-byte words within the env's block of `words` per substep). What the reverse
// cannot cheaply recompute: the substep's input state, the contact and row lists, the joint-space
// factor L, Y = L^-1 J^T, the generalized acceleration and the solve's vectors, and every row
// update's impulse before it and separation used.
struct TapeLayout {
  int words;  // per env and substep (multiple of 4)
  int hdr;    // 4: n_con | n_lim | R | 0 (int bits)
  int st;     // 2 per joint DOF row (q, qd; a ball joint's three rows: rotation vector, angular
              // velocity), then 13 per actor root (p 3 | quat 4 | v 3 | w 3)
  int vec;    // 7 x n: qdd | v_free | z0 = L^T v_free | z final | dz final | v | dq
  int L;      // n x LT (LT = n | 1, odd), row-major, lower triangle
  int Linv;   // n: 1 / L_kk
  int con;    // cw x ccap (SoA): x y z (relative to body a's actor origin) | link a | shape a, and for
              // env types with shape pairs | link b (-1: the ground) | candidate | normal (3, from b
              // to a) | b's actor origin minus a's (3)
  int cw;     // 5, or kTapeConPairWords with shape pairs
  int rowc;   // 4 x rcap: the row headers (16-byte aligned)
  int rowa;   // rcap
  int lam0;   // rcap: warm-start impulses
  int lamf;   // rcap: final impulses
  int lamb;   // (npos + nvel) x rcap: impulse of row r before its update in iteration it
  int seps;   // (npos + 1) x rcap: separation d_r + Y_r . dz used in iteration it (the last for
              // every velocity iteration)
  int Y;      // n x YT (YT = rcap | 1, odd): Y = L^-1 J^T, column r = row r; last, so that a
              // reverse arena without room for it copies the block up to Y and reads Y in place
  int rcap, ccap, n, npos, iters;
  int YT, LT; // odd strides of Y and L (the reverse kernel reads its image in place)
};
constexpr int kTapeConPairWords = 13;

// Arguments of one env type (read once per group, at the start of its step).
struct TypeArgs {
  const EnvTypeTable* type;
  const int* env_ids;        // env ids of the type (nullptr: env_first + index)
  int env_first;
  int n_launch_envs;
  float* scratch;            // lay.scratch_words per group (see the launch wrappers), or null
  SmemLayout lay;
  float* tape;               // taped instantiation only: the type's tape, env-major then substep
  TapeLayout tl;
};

// Shared-memory arena of one env in the reverse (adjoint) kernel, offsets in words. The arena
// starts with an image of the substep's tape block (TapeLayout offsets, copied by one bulk
// asynchronous copy per substep and read in place); the impulses of its final-impulse block are
// rewound in place during the reverse solve.
struct AdjLayout {
  int img;          // the tape block (16-byte aligned): imgw words of it
  int imgw;         // TapeLayout::words, or TapeLayout::lamb when gY
  int gY;           // 1 (env types with shape pairs whose arena would not otherwise fit a CTA's
                    // envs): Y and the row history (lamb, seps) are read in place from the tape, and
                    // Y's adjoint (AdjArgs::ybg) and the row work blocks (AdjArgs::rwg: frw words of
                    // row vectors, then xbw x rcap of xb) live in global slots per group
  int frw, rw;      // gY: words of the row-vector part and of a whole rwg slot
  int bar;          // the bulk copy's mbarrier (8-byte aligned, 4 words reserved)
  int Yb, YS;       // n x YS (YS = the tape's Y stride): Y's adjoint, then the Jacobian-row adjoint
  int Mb, LS;       // n x LS (LS = the tape's L stride): P, then L^-T P, then the inertia adjoint
  int lamb, db, invAb;  // rcap each
  int xb, xbw;      // xbw x rcap: per contact row the adjoint of its contact point (3), and with
                    // shape pairs those of b's actor offset (3) and of its direction (3)
  int vec;          // kAdjVecs x n (see adjoint_kernel.cuh)
  int SD, FM, FMb, Sb;  // 7 x n each (6-vectors at an odd stride): motion subspace, composite-inertia
                        // force, its adjoint, S adjoint
  int link;         // kAdjLinkWords x L
  int pose;         // 12 x L with shape pairs (rotation 9 | origin 3 of each link), else 0 words
  int total;        // words per env (multiple of 4)
};
constexpr int kAdjVecs = 6;
constexpr int kAdjLinkWords = 57;

// Arguments of the reverse pass of one recorded step.
struct AdjArgs {
  const float* tape;         // the type's tape (as written by the taped step)
  const float* g_root;       // (N_A, 13) gradient w.r.t. the step's output root state, or null
  const float* g_dof;        // (N_D, 2) or null
  const float* g_cache;      // (n_envs, cache_stride) or null
  float* gi_root;            // (N_A, 13) out
  float* gi_dof;             // (N_D, 2) out
  float* gi_act;             // (N_D,) out
  float* gi_cache;           // (n_envs, cache_stride) out (also the working storage between substeps)
  int* status;               // (n_envs,) out or null
  float* ybg;                // al.gY: n x YS floats per group of the launch (Y's adjoint), else null
  float* rwg;                // al.gY: al.rw floats per group of the launch (row work blocks), else null
  AdjLayout al;
};

// Persistent heterogeneous launch: one StepArgs per env type plus the tile schedule.
constexpr int kMaxPersistTypes = 8;
enum : int { kVar8 = 0, kVar16 = 1, kVar32 = 2, kVarRowsGlobal = 4 };  // kernel variant codes
struct PersistArgs {
  StepArgs common;
  TypeArgs types[kMaxPersistTypes];
  int variant[kMaxPersistTypes];   // per type: kVar8 / kVar16 / kVar32, | kVarRowsGlobal
  int order[kMaxPersistTypes];     // schedule position -> type
  int tile_end[kMaxPersistTypes];  // inclusive prefix sums of warp tiles in schedule order
  int n_tiles;
  int n_warps;                     // resident warps of the launch
  int warp_words;                  // shared arena words per warp
  unsigned* counter;               // [0] next tile, [1] finished warps (zero between launches)
};

}  // namespace artsim
