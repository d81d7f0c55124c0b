// Host-side symbolic analysis for the fixed-pattern LU of G_k (done once per circuit).
//
// G_k changes value every step but never pattern (the topology is fixed; Alg. 2 factors
// G_k once per step), so ordering, elimination tree, supernodes, the multifrontal
// refactor plan and the triangular-solve task lists are computed here once.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace ers {

struct SymbolicOptions {
  int leaf_size = 32;        // nested-dissection parts at or below this size get minimum degree
  int sep_window_pct = 0;    // 0: separator = the BFS level at the median; w > 0: the smallest
                             // level leaving at least (50 - w)% of the part on each side
  int sep_roots = 1;         // 2: also try the BFS from the other end of the pseudo-diameter
                             // and keep the smaller separator
  int max_width = 64;        // supernode width cap (columns)
  int relax_zeros = 20;      // relaxed amalgamation: max % explicit zeros (0 = fundamental only)
  int relax_width = 16;      // merged supernodes up to this width are accepted regardless
  int solve_chunk = 64;      // rows of the near chunk done by a large supernode's DIAG task
  int warp_chunk = 32;       // rows of a forward far chunk (one warp; 8 chunks per BULK entry)
  int bwd_chunk = 128;       // rows of a backward far chunk (one warp: FMAs over 4 row slabs
                             // before one cross-lane exchange; matches the kernel's BCH)
  int fused_limit = 2048;    // w*(w+r) at or below which one warp does a supernode's solve
  int lane_rows = 32;        // supernodes of at most lane_width columns and lane_rows rows
  int lane_width = 4;        // are solved one per lane (32 per warp task); 0 rows disables
  int lane_min_level = 4096; // ... on levels with at least this many of them (narrower levels
                             // are latency-bound and get a warp per supernode)
  int merge_min_width = 192; // chains of supernodes forming one dense triangular block of at
                             // least this many columns are solved as one merged block through
                             // the explicit inverse of its triangle (0 disables)
  int merge_max_width = 16384;
  int merge_pad_pct = 25;    // explicit zeros allowed to make a near-nested child nest (% of
                             // its own off-diagonal panel)
  int merge_col_block = 8;   // pieces per column block of a merged block's GEMV task
};

// Work entry of the triangular-solve kernels.  A CTA takes one entry at a time:
//   GROUP : up to 8 small supernodes (a..a+b-1 in the small-task list), one per warp;
//   DIAG  : a large supernode's diagonal block plus its nearest row chunk [0, r1);
//   OFF   : a further row chunk [r0, r1) of a large supernode (one warp);
//   BULK  : up to 8 OFF chunks (a..a+b-1 in the chunk list), one per warp.
enum TaskKind : int32_t { TASK_FUSED = 0, TASK_DIAG = 1, TASK_OFF = 2, TASK_GROUP = 3,
                          TASK_BULK = 4, TASK_LANES = 5, TASK_MGEMV = 6 };

struct SolveTask {
  int32_t kind;
  int32_t sn;           // supernode (GROUP: first small task index)
  int32_t r0, r1;       // row range inside R_off(sn) (GROUP: r0 = count)
  int32_t tgt0, ntgt;   // distinct target supernodes of the rows (forward counters)
  int32_t wait_sn;      // backward: supernode whose completion the task waits for
  int32_t wait_cnt;     // forward DIAG/FUSED: arrivals expected; backward DIAG: far chunks
  int32_t c0, w, r;     // the supernode's first column, width and off-diagonal row count
  int32_t grp;          // merged block of the supernode (-1: none); OFF chunks of a merged
                        // piece read z from / accumulate into the block buffer Z
  int64_t d_off, o_off, row_off;  // offsets of its diagonal block, panels and row list
};
// TASK_MGEMV (a CTA entry): one row tile (piece sn) of a merged block times the column pieces
// [r0, r1) of the block's explicit inverse M (lower M_L forward, upper M_U backward):
//   partial = M[rows of sn, columns of r0..r1-1] v, v = y (forward) or Z (backward);
// tgt0 = its partial-sum slot, wait_sn = the first slot of its row tile, wait_cnt = the tasks
// of its row tile, grp = the block, c0 / w = the piece's columns, r = ld of M (the block
// width), d_off = offset of M[row o_sn, column o_r0] in the M storage, o_off = first column of
// the column range, row_off = last column + 1.  The last task of a row tile sums the slots in
// order and writes the tile (Z forward, y backward).

// Inversion job of a merged block (after the refactor): C = alpha op(A) op(B) or a copy.
enum MJobKind : int32_t { MJOB_COPY = 0, MJOB_COPYT = 1, MJOB_GEMM = 2 };
enum MArr : int32_t { MARR_LDI = 0, MARR_UDI = 1, MARR_LO = 2, MARR_UO = 3, MARR_ML = 4,
                      MARR_MU = 5, MARR_SCR = 6 };
enum MTri : int32_t { MTRI_A_LOWER = 1, MTRI_A_UPPER = 2, MTRI_B_LOWER = 4, MTRI_B_UPPER = 8 };
struct MJob {
  int32_t kind, m, n, k;
  int32_t a_arr, b_arr, c_arr, tri;
  int32_t lda, ldb, ldc, pad;
  int64_t a_off, b_off, c_off;
  double alpha;
};

struct Symbolic {
  int n = 0;
  std::vector<int32_t> perm;    // new -> old
  std::vector<int32_t> iperm;   // old -> new
  // permuted pattern of A (G_lin union device stamps), CSR, new indices, rows sorted
  std::vector<int32_t> a_ptr, a_idx;
  std::vector<int32_t> a_src;   // slot in the caller's (old-order) union CSR for each new slot
  // elimination tree (column level)
  std::vector<int32_t> parent;
  std::vector<int64_t> colcount;
  // supernodes
  int nsn = 0;
  std::vector<int32_t> sn_start;   // nsn+1
  std::vector<int32_t> sn_of;      // n
  std::vector<int32_t> sn_parent;  // nsn
  std::vector<int64_t> rptr;       // nsn+1 : R_off(s) = rows[rptr[s] .. rptr[s+1])
  std::vector<int32_t> rows;       // sorted off-diagonal row structure of each supernode
  std::vector<int32_t> rel;        // same layout: position of rows[.] inside the parent's front
  std::vector<int32_t> level;      // multifrontal level (0 = leaves)
  int nlevels = 0;
  // factor storage (doubles)
  std::vector<int64_t> d_off;      // nsn : offset of the w*w inverted diagonal blocks
  std::vector<int64_t> o_off;      // nsn : offset of the r*w off-diagonal panels
  int64_t d_total = 0, o_total = 0;
  // multifrontal plan
  std::vector<int64_t> front_off;  // nsn : offset of the f*f front in the arena (doubles)
  int64_t arena_size = 0;
  std::vector<int32_t> lvl_sn_ptr, lvl_sn;        // supernodes by level
  std::vector<int64_t> asm_dst;                   // per A slot (new order): arena offset
  std::vector<int32_t> lvl_slot_ptr, lvl_slot;    // A slots by level of their supernode
  // extend-add: (child) pairs grouped by (level of parent, child rank)
  std::vector<int32_t> ea_ptr;     // nlevels * maxrank + 1
  std::vector<int32_t> ea_child;
  int ea_maxrank = 0;
  // children of each supernode in rank order (CSR): the per-level extend-add
  std::vector<int32_t> ch_ptr, ch_list;
  // GEMM tile lists per level (Schur update F22 -= F21 F12)
  std::vector<int32_t> tile_ptr;   // nlevels+1
  std::vector<int32_t> tile_sn;    // per tile: supernode
  std::vector<int32_t> tile_ij;    // per tile: (ti << 16) | tj
  // panel-row task lists per level (F21 <- F21 U11^-1, F12 <- L11^-1 F12)
  std::vector<int32_t> ptask_ptr;  // nlevels+1
  std::vector<int32_t> ptask_sn, ptask_r0;
  // triangular solve tasks
  std::vector<SolveTask> fwd, bwd;       // CTA entries, topological order
  std::vector<SolveTask> fwd_small, bwd_small;  // warp tasks referenced by GROUP/BULK entries
  std::vector<int32_t> fwd_tgt;    // target lists of forward tasks
  std::vector<int32_t> fwd_expect; // nsn : units that scatter into each supernode
  std::vector<int32_t> bwd_nchunk; // nsn : far OFF chunks of each supernode (backward)
  // lane items of TASK_LANES warp tasks, 4 ints each: forward (sn, tgt0, ntgt, expected
  // arrivals), backward (sn, parent, 0, 0)
  std::vector<int32_t> fwd_lane, bwd_lane;
  // merged blocks: consecutive supernodes first..last, each the parent of the previous, whose
  // row structures nest (R(s) = columns of s+1 followed by R(s+1)), i.e. one dense W x W
  // triangle; solved through its explicit inverse M (W x W column-major, ld W)
  std::vector<int32_t> grp_first, grp_last, grp_c0, grp_W;
  std::vector<int64_t> grp_moff;   // offset of the block's M in the ML / MU storage
  int64_t m_total = 0;             // doubles of ML (and of MU)
  std::vector<int32_t> sn_grp;     // nsn: block of each supernode (-1: none)
  int32_t nslots = 0;              // partial-sum slots of the MGEMV tasks (per direction)
  // inversion plan: jobs in dependency phases, each phase a list of 64 x 64 output tiles
  std::vector<MJob> mjobs;
  std::vector<int32_t> mphase_ptr; // tiles of phase q: mtile[mphase_ptr[q] .. mphase_ptr[q+1])
  std::vector<int32_t> mtile;      // 2 ints per tile: job, (tile row << 16) | tile column
  int64_t mscratch = 0;            // doubles of scratch the inversion needs
  double minv_flops = 0.0;
  // statistics
  int64_t nnz_L = 0;               // including the diagonal
  double flops = 0.0;              // refactor flops
  int max_front = 0;
  int etree_height = 0;
};

// pattern: n x n CSR (old order, rows sorted, unique). Returns "" on success.
// Check the triangular-solve work lists: every supernode is computed by exactly one task per
// direction, and every wait of a task (forward: the arrivals of all units that scatter into
// it, the DIAG task that publishes a far chunk's supernode; backward: the parent's or the
// touched ancestor's completion, the far chunks a DIAG counts) refers to an entry earlier in
// its list, which makes the persistent solves deadlock-free.  counts[8] receives: forward and
// backward CTA entries, lane items, warp-task supernodes, DIAG entries (fwd, bwd each).
std::string check_solve_plan(const Symbolic& S, int64_t counts[8]);
// Check the inversion plan of the merged blocks: every job stays inside its arrays, the tiles
// of a job cover its output once, and a phase only reads what earlier phases wrote.
std::string check_minv_plan(const Symbolic& S);

std::string analyze(int n, const int32_t* ptr, const int32_t* idx, const SymbolicOptions& opt,
                    Symbolic& out);

}  // namespace ers
