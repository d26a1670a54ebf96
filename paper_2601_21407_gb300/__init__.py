"""GB300-native (sm_103a) Hodgkin-Huxley hot path of BrainFuse.

``hh``      ctypes binding of libhh.so (include/hh.h): networks of HH point
            neurons with user-defined channels, CSR spike propagation with
            delays and exponential synapses, Poisson background.
``inputs``  seeded synthetic workloads and neuron-model tables.
"""
__all__ = ["hh", "inputs"]
