"""GB300-native spatio-temporal LiDAR compression (CUDA kernels for sm_103a behind a C ABI).

``paper_2008_06972_gb300.lcc`` is the ctypes binding of ``include/lcc.h``;
``paper_2008_06972_gb300.build`` compiles ``liblcc.so`` in-tree.  Importing the
package loads nothing: the binding loads the library on first use and fails
loudly if it has not been built.
"""
