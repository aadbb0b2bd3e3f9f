// Launch sequences instantiated for the Minkowski (Cartesian) metric.
#include "hr_run.cuh"
template struct hr::Run<hr::MINK>;
