// Instantiations of the fused kernel for nfft = 1024 .. 4096.
#include "isr_kernels.cuh"

namespace isr {
KernelEntry entry_mid(int log2n, int txt)
{
    switch (log2n) {
    case 10: return entry_for<10>(txt);
    case 11: return entry_for<11>(txt);
    default: return entry_for<12>(txt);
    }
}
}  // namespace isr
