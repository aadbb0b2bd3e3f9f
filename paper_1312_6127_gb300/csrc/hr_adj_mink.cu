// Adjoint of the step instantiated for the Minkowski metric.
#include "hr_adjoint_run.cuh"
template int hr::Run<hr::MINK>::adjoint(harmrad_ctx*, const double*, double*, double*);
