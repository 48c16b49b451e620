/* Plain-C client of the library: compiled with gcc against include/ only and
 * linked to libhologen.so, it calls the entry points that need no GPU. */
#include <stdio.h>
#include <string.h>

#include "hologen.h"
#include "hologen_cnn.h"

int main(void) {
    hg_opts o;
    memset(&o, 0xff, sizeof o);
    hg_opts_default(&o);
    if (hg_opts_size() != sizeof(hg_opts)) return 1;
    if (o.stream != NULL || o.seed != 0 || o.subframes != 24 || o.use_graph != 1 || o.pipeline != -1 ||
        o.autotune != 1 || o.modulated != 0 || o.fresnel != 0.0f || o.amp_clip != 2.0f || o.lt_grow != 10)
        return 2;
    if (!hg_supported_length(1024) || !hg_supported_length(1080) || hg_supported_length(7)) return 3;
    if (strcmp(hg_status_string(HG_OK), "ok") != 0) return 4;
    hg_plan p = NULL;
    hg_slm slm = {HG_SLM_BINARY, 2};
    if (hg_plan_create(&p, 1024, 1024, 0, slm, HG_GS, &o) != HG_ERR_INVALID_ARG || p) return 5;
    if (hg_plan_create(&p, 1024, 7, 1, slm, HG_GS, &o) != HG_ERR_UNSUPPORTED_SIZE || p) return 6;
    if (hg_run(NULL, NULL, NULL, 1, NULL, NULL) != HG_ERR_INVALID_ARG) return 7;
    if (hg_cnn_forward(NULL, NULL, 1, NULL, NULL) != HG_ERR_INVALID_ARG) return 8;
    printf("c abi ok\n");
    return 0;
}
