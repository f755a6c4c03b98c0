// Instantiations of the fused kernel for nfft = 8192.
#include "isr_kernels.cuh"

namespace isr {
KernelEntry entry_8192(int txt) { return entry_for<13>(txt); }
}  // namespace isr
