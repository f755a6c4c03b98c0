// Instantiations of the fused kernel for nfft = 8 .. 512.
#include "isr_kernels.cuh"

namespace isr {
KernelEntry entry_small(int log2n, int txt)
{
    switch (log2n) {
    case 3: return entry_for<3>(txt);
    case 4: return entry_for<4>(txt);
    case 5: return entry_for<5>(txt);
    case 6: return entry_for<6>(txt);
    case 7: return entry_for<7>(txt);
    case 8: return entry_for<8>(txt);
    default: return entry_for<9>(txt);
    }
}
}  // namespace isr
