// Device image layout shared by the host packer and the CUDA kernels.
//
// A packed plan is one contiguous byte image uploaded once into caller-owned device memory:
//   [data]   the applied matrices, in apply order: T~ of every block of levels 0..L (the
//            non-identity part of each interpolative decomposition, Sec. 2) followed by the
//            column bases U_tau of the space leaves; each matrix row-major with its row
//            stride padded to 16 bytes, so every row starts 16-byte aligned;
//   [index]  int32 absolute input indices per block: K entries, skeleton first, then the
//            columns of T~ (level 0: original mode indices; level l >= 1: positions in the
//            level l-1 butterfly vector);
//   [desc]   one MhtBlockDesc per block and stage;
//   [items]  work items (block, first row/column, count) per stage and direction;
//   [perm]   int32 space permutation (tree order -> original point);
//   [weights] w in the apply precision (analysis weights).
#pragma once
#include <stdint.h>

struct MhtBlockDesc {   // 32 bytes
  long long t_off;      // element offset of the block's matrix in [data]
  int ldt;              // row stride in elements (multiple of 16 bytes)
  int rows;             // ID stage: rank r;  U stage: |tau|
  int cols;             // ID stage: K - r;   U stage: r_L
  int idx_off;          // ID stage: offset of the K indices in [index]; U stage: unused
  int out_off;          // ID stage: offset of y_b in this level's vector; U stage: first
                        // tree-order position of tau (into [perm])
  int in_off;           // U stage: offset of y_{tau,root} in the level-L vector
};

struct MhtItem {        // 16 bytes
  int blk;              // block index within the stage
  int start;            // first row (synthesis) or first column (analysis)
  int count;            // rows or columns in this item
  int sib;              // analysis of ID levels >= 1: sibling buffer (tau & 1)
};

struct MhtPItem {       // persistent work item: rows [start, start+count) of one block
  int stage;            // 0..L transfer levels, L+1 column bases
  int blk;
  int start;
  int count;
};

// Batched apply of many plans in one persistent launch: one record per (instance, stage,
// direction) with the device addresses its items read and write, and one item per work
// item of any instance, in dependency order (all items of an instance's phase k precede its
// phase k+1).
struct MhtBatchRec {              // 128 bytes
  unsigned long long data;        // matrices of the instance (its packed image, [data])
  unsigned long long idx;         // its [index]
  unsigned long long desc;        // block descriptors of this stage and direction
  unsigned long long perm;        // its space permutation
  unsigned long long wts;         // its weights (used when the launch asks for weights)
  unsigned long long in0, in1;    // input vector (and sibling buffer for the adjoint)
  unsigned long long out0, out1;  // output vector (and sibling buffer)
  long long is_e, is_k, os_e, os_k;  // element strides (entry, right-hand side)
  int nrhs;
  int mode;                       // 0 synthesis ID, 1 adjoint ID, 2 synthesis U, 3 adjoint U
  int cplx;                       // complex instance (interleaved float pairs)
  int wait_ctr;                   // completion counter to wait for (-1: none)
  unsigned wait_count;            // ... until it reaches this many items
  int done_ctr;                   // counter this record's items increment when done
};

struct MhtBItem {       // 16 bytes
  int rec;              // record index
  int blk;              // block within the record's stage
  int start;            // first row / column
  int count_sib;        // count | (sibling buffer << 31)
};

static_assert(sizeof(MhtBatchRec) == 128, "batch record size");
static_assert(sizeof(MhtBItem) == 16, "batch item size");
static_assert(sizeof(MhtBlockDesc) == 32, "descriptor size");
static_assert(sizeof(MhtPItem) == 16, "persistent item size");
static_assert(sizeof(MhtItem) == 16, "item size");
