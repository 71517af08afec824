// H-matrix block structure and the op programs the planner emits for the
// device interpreter (H-LU factorisation and H-triangular solves, Sec. 4.1).
#pragma once

#include <cstdint>
#include <vector>

#include "hfsem_internal.h"

namespace hf {

// A dense operand inside an instance's arena: stored column-major with
// leading dimension ld; tr = 1 means the logical matrix is the transpose of
// the stored one.  A negative r or c means "the current rank of LR slot
// (-1 - r)", read by the device at execution time.
struct View {
  long long off;
  int r, c;
  int ld;
  int tr;
};

enum OpType : int {
  OP_GEMM = 1,        // C = beta C + alpha A B
  OP_GETRF_INV = 2,   // LU of C (n x n, no pivoting); A <- L^-1, B <- U^-1
  OP_TRMM_L = 3,      // C <- A C   (A square, stored)
  OP_TRMM_R = 4,      // C <- C A
  OP_APPEND = 5,      // LR slot: U += [alpha A], V += [B] (B ident if B.off < 0)
  OP_TRUNC = 6,       // LR slot: recompress to tolerance / rank cap
  OP_ZERO = 7,        // C = 0
  OP_AXPY = 8,        // C += alpha A
};

struct HOp {
  int type;
  int slot;            // LR slot (APPEND / TRUNC)
  double alpha, beta;
  View A, B, C;
};

enum BlkType : int { B_DENSE = 0, B_LR = 1, B_HIER = 2 };

struct Cluster {
  int e0, e1;     // elements [e0, e1)
  int d0, d1;     // element-major unknowns [d0, d1)
  int kid[2];
  int lo, hi;     // support nodes [x_lo, x_hi]
};

struct Block {
  int t, s;           // row / column clusters
  int type;
  int kid[4];         // (t1,s1) (t1,s2) (t2,s1) (t2,s2)
  int m, n;           // rows, cols
  long long off;      // dense: m x n;  LR: U (m x kcap) then V (n x kcap)
  long long inv;      // diagonal dense leaves: L^-1 then U^-1 (n x n each)
  int slot;           // LR slot index
  int kcap, kmax;     // LR capacity / rank cap
  int lower;          // LR: 1 if t is right of s (block of S_l)
};

// A compiled plan for one instance shape.
struct HPlan {
  int N, P, Nd;
  std::vector<Cluster> C;
  std::vector<Block> B;
  std::vector<int> lr_blocks;      // block ids of LR blocks, by slot
  std::vector<int> dense_blocks;   // block ids of dense blocks
  std::vector<HOp> fac;            // H-LU program
  std::vector<HOp> sol;            // forward + backward substitution on the rhs area
  long long arena = 0;             // elements (T) per instance
  long long rhs_off = 0;           // rhs area: Nd x nrhs_max
  int nrhs_max = 0;
  long long ws_off = 0, ws_size = 0;   // truncation workspace
  int kconcat_max = 0;                 // largest rank a truncation sees
  int leaf_max = 0;                    // largest diagonal leaf
  int n_slots = 0;
  int hh_lr = 0;                       // H x H products into LR blocks seen
  long long tmp_base = 0, tmp_size = 0;  // temporaries region
  struct TmpAlloc {
    long long off, size;
    int ld;
  };
  std::vector<TmpAlloc> tmps;          // every temporary handed out
  std::vector<int> fac_waves, sol_waves;   // op offsets of the dependency waves
  int ncta = 1;                        // CTAs that execute one instance
};

struct PlanOpts {
  double lambda;
  int leaf_elems;
  int R;
  int kmax;
  int nrhs_max;
  int max_concat;    // limit on K in a truncation (shared memory)
  int max_leaf;      // limit on diagonal leaf size
  int unique_tmp = 0;  // 1: never reuse temporary storage (independent ops stay independent)
  int ncta = 1;        // CTAs per instance (one truncation workspace each)
};

// Build clusters, blocks, storage and the two programs.
void make_plan(const InstHost& I, const PlanOpts& o, HPlan& out);

}  // namespace hf

namespace hf {
// Dependency levels of an op program: op i may run concurrently with every
// op of the same level; level(i) = 1 + max level of the earlier ops it
// conflicts with (read/write or write/write on overlapping storage, or on the
// same low-rank slot / rank).  Returns the number of levels.
int program_levels(const HPlan& p, const std::vector<HOp>& prog, std::vector<int>& level);

// Split large ops into independent tile ops, then order the program by
// dependency level; waves[w] .. waves[w+1] are the ops of wave w.
void schedule_program(const HPlan& p, std::vector<HOp>& prog, std::vector<int>& waves);
}  // namespace hf
