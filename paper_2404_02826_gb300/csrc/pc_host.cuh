// Host-side switches of the entry points.  Internal.
#pragma once

namespace pcx {

// While on for the calling host thread, the library allocates nothing on the
// host side: read-backs use page-locked staging blocks that already exist, else
// go straight to their destinations, and the bit-box reduction issues its
// rounds one launch at a time instead of capturing a CUDA graph
// (pc_compress_noalloc, whose callers may not allocate).
void set_no_host_alloc(bool on);
bool no_host_alloc();  // the calling thread's switch

}  // namespace pcx
