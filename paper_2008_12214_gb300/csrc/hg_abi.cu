// hg_abi.cu -- layout check of the option structure for bindings.
#include "hologen.h"

extern "C" size_t hg_opts_size(void) { return sizeof(hg_opts); }
