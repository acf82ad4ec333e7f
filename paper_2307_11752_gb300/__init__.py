"""GB300-native lattice Boltzmann BGK collide-and-stream (D2Q9 / D3Q19).

The compute path is the CUDA library ``libolb.so`` behind the C ABI declared in
``include/olb.h``.  ``paper_2307_11752_gb300.olb`` is its ctypes binding (import
it explicitly); ``paper_2307_11752_gb300.opti`` identifies porosity fields with
the GPU adjoint and torch's L-BFGS; ``paper_2307_11752_gb300.inputs`` builds
seeded synthetic workloads and needs no GPU.
"""
