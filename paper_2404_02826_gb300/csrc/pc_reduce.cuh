// Declarations of the bit-box reduction (csrc/k_reduce.cu) for the compress
// driver.  Nothing here is part of the public C ABI (include/pc.h).
#pragma once

#include "pc_internal.cuh"

namespace pcx {

// Bit-box reduction (Sec. 4.1, Alg. 1) over the leaves of the last level.
struct ReduceLaunch {
  uint64_t n;
  int code_bytes;
  int split_level;
  uint32_t leaf_size;
  uint64_t num_leaves;
  const void *codes[3];     // leaf-ordered codes
  const uint32_t *idx;      // leaf-ordered input indices (optional)
  void *out_codes[3];       // codes in sequence order (written)
  uint32_t *out_idx;        // input indices in sequence order (written when idx is given)
  LeafRec *leafs;           // [num_leaves] scratch: the leaf ranges
  LeafRec *seqs;            // [num_leaves] the sequences: off, cnt, centre = 0, m, q_ref, words
  void *scratch;            // reduce_scratch_bytes(n, num_leaves), 256-byte aligned
  uint32_t *err;
};
uint64_t reduce_scratch_bytes(uint64_t n, uint64_t num_leaves);
// Runs the rounds (reading a counter back every few rounds); on success
// *num_seq holds the number of sequences and *rounds the rounds taken.
cudaError_t launch_reduce(const ReduceLaunch &a, cudaStream_t st, uint64_t *num_seq, uint64_t *rounds);

}  // namespace pcx
