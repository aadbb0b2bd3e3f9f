// Launch sequences instantiated for the Kerr-Schild metric.
#include "hr_run.cuh"
template struct hr::Run<hr::KS>;
