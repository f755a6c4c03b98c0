// Instantiations of the fused kernel for nfft = 16384 (the paper's transform length).
#include "isr_kernels.cuh"

namespace isr {
KernelEntry entry_16384(int txt) { return entry_for<14>(txt); }
}  // namespace isr
