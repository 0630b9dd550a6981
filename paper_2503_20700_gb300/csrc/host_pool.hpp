// Persistent host worker threads for the planning passes of a bond (operator
// placement lists, H_eff psi item lists, tcgen05 task lists).  run(n, fn)
// calls fn(i) once for every i in [0, n), on the workers and the calling
// thread, taking indices from a shared counter; it returns when every call
// has finished.  Callers that need a deterministic result write the result
// of index i to slot i and merge the slots in index order.
#pragma once
#include <cstddef>
#include <functional>

namespace dmrg {

void host_parallel_for(size_t n, const std::function<void(size_t)>& fn);

// threads taking part in host_parallel_for (workers + the caller)
unsigned host_threads();

}  // namespace dmrg
