/* Prints the size of every struct that include/isr.h declares and the offset of each of
 * its fields, one "struct.field offset" line each, so a test can compare the C layout
 * with the ctypes mirror of the Python binding.  Compiled as C (not C++) against the
 * public header only. */
#include <stddef.h>
#include <stdio.h>

#include "isr.h"

#define SIZE(T) printf("%s size %zu\n", #T, sizeof(T))
#define FIELD(T, f) printf("%s.%s %zu\n", #T, #f, offsetof(T, f))

int main(void)
{
    SIZE(isr_plan_desc);
    FIELD(isr_plan_desc, nfft);
    FIELD(isr_plan_desc, code_len);
    FIELD(isr_plan_desc, n_ranges);
    FIELD(isr_plan_desc, range_start);
    FIELD(isr_plan_desc, range_step);
    FIELD(isr_plan_desc, tx_type);
    FIELD(isr_plan_desc, echo_stride);
    FIELD(isr_plan_desc, tx_stride);
    FIELD(isr_plan_desc, ipp_chunk);
    FIELD(isr_plan_desc, max_chunks);
    FIELD(isr_plan_desc, device);
    FIELD(isr_plan_desc, flags);
    FIELD(isr_plan_desc, stream);

    SIZE(isr_ranges);
    FIELD(isr_ranges, start);
    FIELD(isr_ranges, step);
    FIELD(isr_ranges, count);

    SIZE(isr_plan_info);
    FIELD(isr_plan_info, nfft);
    FIELD(isr_plan_info, n_ranges);
    FIELD(isr_plan_info, ranges_per_cta);
    FIELD(isr_plan_info, threads_per_cta);
    FIELD(isr_plan_info, smem_bytes);
    FIELD(isr_plan_info, max_chunks);
    FIELD(isr_plan_info, ipp_chunk);
    FIELD(isr_plan_info, sm_count);
    FIELD(isr_plan_info, n_ipp_integrated);
    FIELD(isr_plan_info, kernel_launches);
    FIELD(isr_plan_info, kernel_ms);
    FIELD(isr_plan_info, kernel_timed);
    FIELD(isr_plan_info, host_block_growth);

    SIZE(isr_window);
    FIELD(isr_window, echo);
    FIELD(isr_window, tx_code);
    FIELD(isr_window, out);
    FIELD(isr_window, echo_stride);
    FIELD(isr_window, tx_stride);
    FIELD(isr_window, nfft);
    FIELD(isr_window, code_len);
    FIELD(isr_window, n_ranges);
    FIELD(isr_window, range_start);
    FIELD(isr_window, range_step);
    FIELD(isr_window, n_ipp);
    FIELD(isr_window, order);
    FIELD(isr_window, reserved);

    SIZE(isr_batch_info);
    FIELD(isr_batch_info, n_windows);
    FIELD(isr_batch_info, graph);
    FIELD(isr_batch_info, n_units);
    FIELD(isr_batch_info, transforms);
    FIELD(isr_batch_info, order);
    FIELD(isr_batch_info, tune_ms);
    return 0;
}
