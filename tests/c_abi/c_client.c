/* A plain C user of the library: create a plan, integrate host-resident IPPs, read the
 * spectra into host memory, destroy the plan -- the calls of the C ABI in include/isr.h,
 * with no Python in between.
 *
 *   c_client ECHO CODE OUT NFFT N_RANGES RANGE_STEP N_IPP ECHO_STRIDE
 *
 * ECHO: raw int16 [N_IPP][ECHO_STRIDE][2]; CODE: raw int8 [NFFT] (binary phase);
 * OUT: written as raw float [N_RANGES][NFFT] (the sums over IPPs).  The IPPs are added in
 * two calls to check that repeated calls continue one integration.  Exit status 0 on
 * success; on failure the status name and isr_last_error() go to stderr. */
#include <stdio.h>
#include <stdlib.h>

#include "isr.h"

static void* read_all(const char* path, size_t bytes)
{
    FILE* f = fopen(path, "rb");
    if (!f) return NULL;
    void* buf = malloc(bytes ? bytes : 1);
    size_t got = buf ? fread(buf, 1, bytes, f) : 0;
    fclose(f);
    if (got != bytes) {
        free(buf);
        return NULL;
    }
    return buf;
}

static int check(isr_status st, const char* what)
{
    if (st == ISR_OK) return 0;
    fprintf(stderr, "%s failed with status %d: %s\n", what, (int)st, isr_last_error());
    return 1;
}

int main(int argc, char** argv)
{
    if (argc != 9) {
        fprintf(stderr, "usage: %s ECHO CODE OUT NFFT N_RANGES RANGE_STEP N_IPP ECHO_STRIDE\n", argv[0]);
        return 2;
    }
    const int nfft = atoi(argv[4]), n_ranges = atoi(argv[5]), step = atoi(argv[6]), n_ipp = atoi(argv[7]);
    const long long stride = atoll(argv[8]);
    const size_t echo_bytes = (size_t)n_ipp * (size_t)stride * 4;
    int16_t* echo = (int16_t*)read_all(argv[1], echo_bytes);
    int8_t* code = (int8_t*)read_all(argv[2], (size_t)nfft);
    float* out = (float*)malloc((size_t)n_ranges * nfft * sizeof(float));
    if (!echo || !code || !out) {
        fprintf(stderr, "cannot read the inputs\n");
        return 2;
    }

    isr_plan_desc d = {0};
    d.nfft = nfft;
    d.code_len = nfft;
    d.n_ranges = n_ranges;
    d.range_start = 0;
    d.range_step = step;
    d.tx_type = ISR_TX_PM1;
    d.echo_stride = stride;
    d.tx_stride = 0;
    d.device = 0;
    d.stream = NULL;

    isr_plan* plan = NULL;
    int rc = check(isr_plan_create(&plan, &d), "isr_plan_create");
    const int first = n_ipp / 3;
    if (!rc) rc = check(isr_integrate(plan, echo, code, first, NULL, nfft), "isr_integrate (first part)");
    if (!rc)
        rc = check(isr_integrate(plan, echo + (size_t)first * (size_t)stride * 2, code, n_ipp - first, NULL, nfft),
                   "isr_integrate (second part)");
    int64_t n_done = -1;
    if (!rc) rc = check(isr_spectra(plan, out, 0, &n_done), "isr_spectra");
    if (!rc && n_done != n_ipp) {
        fprintf(stderr, "isr_spectra reports %lld IPPs, expected %d\n", (long long)n_done, n_ipp);
        rc = 1;
    }
    isr_destroy(plan);
    if (!rc) {
        FILE* f = fopen(argv[3], "wb");
        if (!f || fwrite(out, sizeof(float), (size_t)n_ranges * nfft, f) != (size_t)n_ranges * nfft) rc = 2;
        if (f) fclose(f);
    }
    free(echo);
    free(code);
    free(out);
    return rc;
}
