"""GB300-native object-centric Census Template Matching (arXiv 2604.07980, Sec. 4.3).

The compute path is the CUDA library ``libctm.so`` (sources in ``csrc/``, C ABI in
``include/ctm.h``); ``paper_2604_07980_gb300.binding`` marshals arguments into it.
``paper_2604_07980_gb300.workloads`` makes seeded synthetic inputs.  Importing the
package itself loads nothing; the binding loads the library on first use and
raises if it is missing.
"""
