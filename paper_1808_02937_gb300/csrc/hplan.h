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
  int kest;            // APPEND / TRUNC: the planner's estimate of the rank the slot
                       // reaches (scheduling only; the device reads ranks at run time)
  int pad;
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
  std::vector<int> fac_waves;          // op offsets of the dependency waves
  int ncta = 1;                        // CTAs that execute one instance
  int R = 0;                           // rank of the Taylor factors
};

// Capacity of a low-rank block in multiples of kmax: updates are appended
// until the capacity is reached, then the block is recompressed (fewer,
// larger recompressions for a larger multiple).
constexpr int kKcapMult = 2;

struct PlanOpts {
  double lambda;       // admissibility parameter of eq. (admis)
  int leaf_elems;
  int R;
  int kmax;
  int nrhs_max;
  int max_concat;    // limit on K in a truncation (shared memory)
  int max_leaf;      // limit on diagonal leaf size
  int unique_tmp = 0;  // 1: never reuse temporary storage (independent ops stay independent)
  int ncta = 1;        // CTAs per instance (one truncation workspace each)
  int structure_only = 0;  // 1: clusters, blocks and storage only (no H-LU program)
  int adm_min = 0;     // 0: max(diam tau, diam sigma) <= lambda dist (eq. (admis));
                       // 1: min(...) <= lambda dist, the expansion being taken
                       // about the smaller cluster (Remark after the Lemma)
};

// Build clusters, blocks, storage and the two programs.
void make_plan(const InstHost& I, const PlanOpts& o, HPlan& out);

}  // namespace hf

namespace hf {
// Triangular solves by leaf clusters (gather form).  Forward, for the leaves
// i in order: x_i = L_ii^-1 (b_i - sum_{j<i} L_ij x_j), where a dense block
// contributes A x_s directly and a low-rank block U V^T contributes U w with
// w = V^T x_s accumulated leaf by leaf as x_s is produced; backward the same
// with U and the leaves in reverse order.  A step (one leaf, one direction)
// is cut into column jobs, each one column segment of a factor restricted to
// the leaf's rows, spread over the CTAs of the instance's cluster:
//   kind 0: r_part += A(:, k) x_s[k]        (dense block column, x_s[k] in
//                                            the ring of recent leaves)
//   kind 4: the same with x_s[k] read from the rhs area
//   kind 1: r_part += U(:, l) w[l]          (low-rank block column, l < rank)
//   kind 2: x_part += D^-1(:, k) r[k]       (inverse diagonal block column)
//   kind 3: w[l]  += V(:, l)^T x            (low-rank column, l < rank)
// The gather and scatter jobs of a low-rank column always go to the same CTA,
// which keeps its w.
struct SolJob {
  long long src;      // first entry of the segment (instance arena offset)
  int x;              // kind 0: ring offset; 4: unknown index; 1, 3: w column of
                      // the owning CTA; 2: k
  int slot;           // kinds 1, 3: LR slot whose rank bounds l; else -1
  short l, kind;
  int ldw;            // kinds 1, 3: leading dimension of w
  int n;              // segment length (the leaf's unknowns)
  int lmax;           // kinds 1, 3: columns the solve reads of the block
};

struct StepInfo {
  int d0, n;          // unknowns of the leaf
  int ring;           // slot of the leaf's solution in the ring of recent leaves
};

struct StepCta {      // jobs of one CTA in one step: [a0, a1) gathers,
  int a0, a1, a2, a3; // [a1, a2) inverse columns, [a2, a3) scatters; they reach
};                    // shared memory in parts of jcap jobs from a0 on

constexpr int kRing = 4;     // leaves whose solutions every CTA keeps

struct LeafSolve {
  std::vector<StepInfo> steps;   // 2 x leaves steps: forward, then backward
  std::vector<StepCta> step_cta; // [step][ncta]
  std::vector<SolJob> jobs;
  int wcols = 1;                 // most low-rank columns one CTA owns
  int jcap = 1;                  // jobs per part
  int nmax = 0;                  // largest leaf
};

// Tables of the leaf solves of a factored plan, for ncta CTAs per instance,
// entries of ts bytes and sw right-hand sides per pass; parts are cut so that
// the solve kernel's shared memory (solve_smem) stays within budget bytes.
// The budget is checked for leaves of at least nmax_min entries and at least
// wcols_min low-rank columns per CTA (when one kernel serves several plans).
void build_leaf_solve(const HPlan& p, int ncta, size_t budget, int ts, int sw, LeafSolve& out,
                      int nmax_min = 1, int wcols_min = 1);

// Shared memory of the leaf-solve kernel for parts of jmax jobs.
size_t solve_smem(int jmax, int nmax, int wcols, int ts, int sw);

// Dependency levels of an op program: op i may run concurrently with every
// op of the same level; level(i) = 1 + max level of the earlier ops it
// conflicts with (read/write or write/write on overlapping storage, or on the
// same low-rank slot / rank).  Returns the number of levels.
int program_levels(const HPlan& p, const std::vector<HOp>& prog, std::vector<int>& level);

// Split large ops into independent tile ops, then order the program by
// dependency level; waves[w] .. waves[w+1] are the ops of wave w, longest
// (by a cost model) first.
void schedule_program(const HPlan& p, std::vector<HOp>& prog, std::vector<int>& waves);
}  // namespace hf
