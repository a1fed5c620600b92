"""GB300-native spectral hyper-viscosity solver for 3D incompressible flow.

The compute path is the CUDA library ``libns3d.so`` behind the C ABI in
``include/ns3d.h``; ``binding`` marshals arguments to it (PyTorch tensors for
device memory and streams).  Importing this package loads nothing; call
``binding.load()`` (or create a ``binding.Plan``) to load the library, which
raises if it has not been built.
"""
__all__ = ["binding", "build"]
