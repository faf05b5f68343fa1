// Kernel selection for a plan: the specialised kernel for (N, T, dtype) when
// one is compiled in, otherwise an empty entry (the plan then uses the general
// kernel, which handles every supported size).
#include "ppf_launch.h"

namespace ppf {

KernelEntry ring_entry(int N, int T, int dtype);  // ppf_ring.cu

KernelEntry select_fast_entry(int N, int T, int dtype)
{
    KernelEntry e = ring_entry(N, T, dtype);
    if (e.launch) return e;
    return KernelEntry{};
}

}  // namespace ppf
