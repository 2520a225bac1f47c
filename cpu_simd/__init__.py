"""CPU comparison baseline: the pi/12 method vectorised across angles on the
host cores (libptrig_cpu, include/ptrig_cpu.h).  Not used by the GPU path."""
