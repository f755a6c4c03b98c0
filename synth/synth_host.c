/*
 * synth_host.c -- host (gcc) build of the seeded synthetic echo generator.
 * All arithmetic is in synth_core.h; this file only loops over rows and samples.
 * Compiled with -ffp-contract=off so its samples match the device build bit for bit.
 */
#include <stdlib.h>
#include <string.h>
#include "synth_core.h"

#ifdef _OPENMP
#include <omp.h>
#endif

void syn_philox_kat(const uint32_t ctr[4], uint64_t seed, uint32_t out[4])
{
    syn_philox(ctr, seed, out);
}

void syn_fill_table(float* table)
{
    for (int j = 0; j < SYN_TABLE_SIZE; ++j) syn_table_entry(j, &table[2 * j], &table[2 * j + 1]);
}

/* code rows [row_begin, row_end) of code_len chips each */
void syn_fill_code(uint64_t seed, int code_len, int row_begin, int row_end, int8_t* code)
{
    for (int q = row_begin; q < row_end; ++q)
        for (int k = 0; k < code_len; ++k)
            code[(size_t)(q - row_begin) * (size_t)code_len + (size_t)k] = (int8_t)syn_code_chip(seed, k, q);
}

void syn_tone_freqs(uint64_t seed, int n, double* out)
{
    for (int r = 0; r < n; ++r) out[r] = syn_tone_freq(seed, r);
}

/* amp_gate: per-gate amplitude, or NULL for c->amp everywhere */
void syn_fill_params(const syn_cfg* c, const double* f_base, const double* amp_gate, int p, syn_rp* out)
{
    for (int r = 0; r < c->n_ranges; ++r)
        out[r] = syn_range_params(c, f_base[r], amp_gate ? amp_gate[r] : c->amp, r, p);
}

/*
 * Echo rows [row_begin, row_end) into out[(p - row_begin)][echo_stride][2].
 * amp_gate: per-gate amplitude or NULL (c->amp for every gate).
 * code: [1][code_len] when per_ipp_code == 0, else rows indexed by absolute p
 *       ([row_end][code_len] at least).
 * Returns 0, or 2 on allocation failure.
 */
int syn_echo_rows(const syn_cfg* c, const double* f_base, const double* amp_gate, const int8_t* code,
                  int64_t row_begin, int64_t row_end, int16_t* out, int n_threads)
{
    float* table = (float*)malloc(sizeof(float) * 2 * SYN_TABLE_SIZE);
    if (!table) return 2;
    syn_fill_table(table);
    int fail = 0;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
    for (int64_t p = row_begin; p < row_end; ++p) {
        syn_rp* rp = (syn_rp*)malloc(sizeof(syn_rp) * (size_t)(c->n_ranges > 0 ? c->n_ranges : 1));
        if (!rp) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            fail = 1;
            continue;
        }
        syn_fill_params(c, f_base, amp_gate, (int)p, rp);
        const int8_t* crow = code + (c->per_ipp_code ? (size_t)p * (size_t)c->code_len : 0);
        int16_t* row = out + (size_t)(p - row_begin) * (size_t)c->echo_stride * 2;
        for (int64_t t = 0; t < c->echo_stride; ++t)
            syn_sample(c, rp, crow, table, t, (int)p, &row[2 * t], &row[2 * t + 1]);
        free(rp);
    }
    free(table);
    return fail ? 2 : 0;
}
