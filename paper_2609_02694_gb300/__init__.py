"""GB300-native improved random batch Ewald (RBE) nonbonded force path.

`binding` wraps the C-ABI shared library (built from `csrc/` by `build`); `synth` draws
seeded synthetic inputs. Importing the package does not load the CUDA library.
"""
