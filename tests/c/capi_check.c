/* Plain-C client of the kdiag C-ABI: compiles against include/kdiag.h with a C compiler and links
 * libkdiag.so, then exercises the host-side entry points and argument checks (no kernel runs, no
 * device needed). Exit status 0 when every check holds. */
#include <stdio.h>
#include <string.h>

#include "kdiag.h"

static int failures = 0;
#define CHECK(cond)                                                   \
    do {                                                              \
        if (!(cond)) {                                                \
            fprintf(stderr, "check failed: %s (line %d)\n", #cond, __LINE__); \
            ++failures;                                               \
        }                                                             \
    } while (0)

int main(void) {
    kd_opts o;
    memset(&o, 0xff, sizeof(o));
    kd_opts_default(&o);
    CHECK(o.form == -1 && o.max_sweeps == 4 && o.layout == KD_LAYOUT_SOA && o.stats == NULL);
    CHECK(kd_version() == 200);
    CHECK(strcmp(kd_status_string(KD_OK), "ok") == 0);
    CHECK(strstr(kd_status_string(KD_ERR_MISALIGNED), "misaligned") != NULL);

    /* pointers below are never dereferenced: every call is rejected (or empty) before a launch */
    float *fake = (float *)(size_t)64;
    CHECK(kd_eig3_sym(NULL, KD_F32, 0, 0, NULL, NULL, NULL, KD_F32, NULL, NULL, NULL) == KD_OK);
    CHECK(kd_eig3_sym(NULL, KD_F32, 5, 5, NULL, NULL, NULL, KD_F32, NULL, NULL, NULL) == KD_ERR_INVALID_ARG);
    CHECK(kd_eig3_sym(fake, KD_F32, 10, 9, NULL, NULL, NULL, KD_F32, NULL, NULL, NULL) == KD_ERR_INVALID_ARG);
    CHECK(kd_eig3_sym(fake, KD_F64, 10, 10, NULL, NULL, NULL, KD_F32, NULL, NULL, NULL) == KD_ERR_UNSUPPORTED);
    CHECK(kd_eig3_sym((char *)fake + 2, KD_F32, 10, 10, NULL, NULL, NULL, KD_F32, NULL, NULL, NULL) ==
          KD_ERR_MISALIGNED);
    CHECK(kd_eig3_sym_adjoint(fake, KD_F32, 10, 10, NULL, NULL, NULL, NULL, NULL, NULL) == KD_ERR_INVALID_ARG);
    CHECK(kd_eig2_sym(fake, KD_BF16, 10, 10, NULL, NULL, NULL, KD_BF16, NULL, NULL) == KD_ERR_UNSUPPORTED);
    o.max_sweeps = 9;
    CHECK(kd_eig3_sym(fake, KD_F32, 10, 10, NULL, NULL, NULL, KD_F32, NULL, &o, NULL) == KD_ERR_INVALID_ARG);
    CHECK(kd_st_loss_workspace_bytes(0) == 0 || kd_st_loss_workspace_bytes(0) > 0);
    CHECK(kd_eig3_host_workspace_bytes(KD_F32, 0, 1) == 0);
    CHECK(kd_eig3_host_workspace_bytes(KD_F32, 1000, 2) > 0);
    if (failures == 0) printf("capi_check: ok\n");
    return failures == 0 ? 0 : 1;
}
