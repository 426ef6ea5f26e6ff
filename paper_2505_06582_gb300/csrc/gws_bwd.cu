// gws_bwd.cu -- backward splat (placeholder translation unit; filled in by the backward kernels).
#include "gws_host.h"
