// isr_kernels.cuh -- kernel registry shared by the instantiation units and the host API.
#pragma once

#include "isr.h"
#include "isr_kernel.cuh"
#include "isr_paired.cuh"

namespace isr {

// record a one-line reason for isr_last_error() and return st (defined in isr_api.cu)
isr_status fail(isr_status st, const char* fmt, ...);
void clear_error();

// radix orders: 0-2 Stockham, 3 warp-local, 4-5 paired FP32, 6-8 orders 0-2 with the inter-pass
// twiddles in tensor memory, 9 the warp-local schedule with its twiddles in tensor memory
constexpr int kNumOrders = 10;

struct KernelEntry {
    const void* fn;   // __global__ integrate_kernel<LOG2N, TXT>
    const void* fn_full;  // the same for code_len == nfft (binary-phase codes only; else fn)
    const void* fn_order[kNumOrders];  // fn_full with radix order 0..8 (1-3: nfft >= 2048; 4-8: 16384)
    int smem_order[kNumOrders];        // their shared memory
    const void* fn_tc[9];     // [mode] tensor-core first pass (nfft 16384, binary phase): 1-4 mma.sync,
                              // 5-8 tcgen05; [0] unused
    int smem_tc;
    int smem;         // dynamic shared memory bytes
    int gates;        // range gates per CTA (G)
    int threads;      // threads per CTA
};

template <int L>
KernelEntry entry_for(int txt)
{
    using S = Sched<L>;
    const void* f = txt == TX_CI16 ? (const void*)integrate_kernel<L, TX_CI16>
                  : txt == TX_C32  ? (const void*)integrate_kernel<L, TX_C32>
                                   : (const void*)integrate_kernel<L, TX_PM1>;
    const void* ff = txt == TX_PM1 ? (const void*)integrate_kernel<L, TX_PM1, true> : f;
    KernelEntry e{f, ff, {ff, ff, ff, ff, ff, ff, ff, ff, ff, ff},
                  {S::SMEM, S::SMEM, S::SMEM, S::SMEM, S::SMEM, S::SMEM, S::SMEM, S::SMEM, S::SMEM, S::SMEM},
                  {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr},
                  0, S::SMEM, S::G, kThreads};
    if constexpr (L >= 11) {
        if (txt == TX_PM1) {
            e.fn_order[1] = (const void*)integrate_kernel<L, TX_PM1, true, 1>;
            e.fn_order[2] = (const void*)integrate_kernel<L, TX_PM1, true, 2>;
            e.fn_order[3] = (const void*)integrate_kernel_wl<L, TX_PM1, true>;
            e.smem_order[1] = Sched<L, 1>::SMEM;
            e.smem_order[2] = Sched<L, 2>::SMEM;
            e.smem_order[3] = SchedWL<L>::SMEM;
        }
    }
    if constexpr (L == 14) {
        if (txt == TX_PM1) {
            e.fn_order[4] = (const void*)integrate_kernel_p<true>;
            e.smem_order[4] = SchedP::SMEM;
            e.fn_order[5] = (const void*)integrate_kernel_q<true>;
            e.smem_order[5] = SchedQ::SMEM;
            e.fn_order[6] = (const void*)integrate_kernel_tm<14, TX_PM1, true, 0>;
            e.smem_order[6] = Sched<14, 0, true>::SMEM;
            e.fn_order[7] = (const void*)integrate_kernel_tm<14, TX_PM1, true, 1>;
            e.smem_order[7] = Sched<14, 1, true>::SMEM;
            e.fn_order[8] = (const void*)integrate_kernel_tm<14, TX_PM1, true, 2>;
            e.smem_order[8] = Sched<14, 2, true>::SMEM;
            e.fn_order[9] = (const void*)integrate_kernel_wl_tm<14, TX_PM1, true>;
            e.smem_order[9] = SchedWL<14>::SMEM;
            e.fn_tc[1] = (const void*)integrate_kernel<14, TX_PM1, true, 1, P0_BF16_SPLIT>;
            e.fn_tc[2] = (const void*)integrate_kernel<14, TX_PM1, true, 1, P0_FP16_SPLIT>;
            e.fn_tc[3] = (const void*)integrate_kernel<14, TX_PM1, true, 1, P0_BF16>;
            e.fn_tc[4] = (const void*)integrate_kernel<14, TX_PM1, true, 1, P0_FP16>;
            e.fn_tc[5] = (const void*)integrate_kernel_tc05<P0_TC05_BF16_SPLIT>;
            e.fn_tc[6] = (const void*)integrate_kernel_tc05<P0_TC05_FP16_SPLIT>;
            e.fn_tc[7] = (const void*)integrate_kernel_tc05<P0_TC05_BF16>;
            e.fn_tc[8] = (const void*)integrate_kernel_tc05<P0_TC05_FP16>;
            e.smem_tc = Sched<14, 1>::SMEM + kTcAfragBytes;
        }
    }
    return e;
}

// defined in the instantiation units (one per group of sizes, compiled in parallel)
KernelEntry entry_small(int log2n, int txt);  // nfft 8 .. 512
KernelEntry entry_mid(int log2n, int txt);    // nfft 1024 .. 4096
KernelEntry entry_8192(int txt);
KernelEntry entry_16384(int txt);

inline KernelEntry kernel_entry(int log2n, int txt)
{
    if (log2n <= 9) return entry_small(log2n, txt);
    if (log2n <= 12) return entry_mid(log2n, txt);
    if (log2n == 13) return entry_8192(txt);
    return entry_16384(txt);
}

}  // namespace isr
