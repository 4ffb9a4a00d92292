// Declarations of the reordering for the entropy coder (csrc/k_reorder.cu)
// for the compress driver.  Nothing here is part of the public C ABI.
#pragma once

#include "pc_internal.cuh"

namespace pcx {

// Sec. 4.2 (after Fig. 4): sequences in increasing sum of m_d, and within
// each sequence (centre first) the particles in increasing R-index.
struct ReorderLaunch {
  uint64_t n;
  int code_bytes;
  uint64_t num_seq;
  const LeafRec *recs;   // [num_seq] off, cnt, centre (position within the sequence), m, q_ref
  LeafRec *out_recs;     // [num_seq] the new order: off, cnt, centre = 0, m, q_ref, words
  const void *codes[3];  // codes at the positions recs describe
  const uint32_t *idx;   // input indices beside them (optional)
  void *out_codes[3];    // codes at their new positions (written)
  uint32_t *out_idx;     // input indices at their new positions (written when idx is given)
  uint64_t max_cnt;      // a bound on the particles of one sequence (sizes the scratch)
  void *scratch;         // reorder_scratch_bytes(n, num_seq, max_cnt), 256-byte aligned
};
uint64_t reorder_scratch_bytes(uint64_t n, uint64_t num_seq, uint64_t max_cnt);
cudaError_t launch_reorder(const ReorderLaunch &a, cudaStream_t st);

}  // namespace pcx
