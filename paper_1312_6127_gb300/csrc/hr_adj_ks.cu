// Adjoint of the step instantiated for the Kerr-Schild metric.
#include "hr_adjoint_run.cuh"
template int hr::Run<hr::KS>::adjoint(harmrad_ctx*, const double*, double*, double*);
