/* A plain C99 user of the C ABI: compiled against include/lbm.h and linked
 * against the library, it exercises the calls that need no GPU (argument
 * checks, error text, host-side sizes) and exits 0 when each behaves as the
 * header states. */
#include <stdio.h>
#include <string.h>

#include "lbm.h"

static int failures = 0;

static void expect(int cond, const char *what)
{
    if (!cond) {
        fprintf(stderr, "FAILED: %s\n", what);
        ++failures;
    }
}

int main(void)
{
    lbm_ctx *ctx = (lbm_ctx *)&failures; /* must be reset to NULL on failure */
    expect(lbm_create(0, 4, 4, LBM_D3Q19, LBM_F32, NULL, NULL, &ctx) == LBM_ERR_ARG, "nx = 0 rejected");
    expect(ctx == NULL, "no context after a failed create");
    expect(strlen(lbm_last_error(NULL)) > 0, "error text for a call without a context");
    ctx = NULL;
    expect(lbm_create(8, 8, 8, (lbm_lattice)15, LBM_F32, NULL, NULL, &ctx) == LBM_ERR_ARG, "D3Q15 rejected");
    expect(lbm_create_ex(8, 8, 8, LBM_D3Q27, LBM_F16_SHIFTED, (lbm_pattern)3, NULL, NULL, &ctx) == LBM_ERR_ARG,
           "unknown pattern rejected");
    expect(lbm_step(NULL, 1) == LBM_ERR_ARG, "step without a context");
    expect(lbm_destroy(NULL) == LBM_OK, "destroy(NULL) is a no-op");
    {
        lbm_reduction r;
        expect(lbm_reduce(NULL, &r) == LBM_ERR_ARG, "reduce without a context");
    }
    {
        char buf[16];
        int layout = -1;
        long long steps = -1;
        expect(lbm_get_state(NULL, buf, sizeof buf, &layout, &steps, 0) == LBM_ERR_ARG, "get_state without a context");
        expect(layout == -1 && steps == -1, "outputs untouched on failure");
    }
    expect(lbm_mlp_workspace_bytes(0) == 0, "no workspace for no samples");
    expect(lbm_mlp_workspace_bytes(100000) > 0, "workspace for samples");
    expect(LBM_NTAGS == LBM_TAG_WALL0 + LBM_NWALLS, "tag count");
    if (failures == 0) printf("abi_host: ok\n");
    return failures == 0 ? 0 : 1;
}
