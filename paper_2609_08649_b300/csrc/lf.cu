// Unity build of the library: one translation unit, so the device error word and the
// helpers are single definitions without relocatable device code.
#include <type_traits>
#include "lf_host.cu"
#include "lf_grid.cu"
#include "lf_hostio.cu"
#include "lf_finder.cu"
#include "lf_trace.cu"
#include "lf_chi2.cu"
#include "lf_sampler.cu"
#include "lf_optimizer.cu"
#include "lf_static.cu"
#include "lf_probe.cu"
