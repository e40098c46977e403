"""GB300-native SR-CPM electrode-charge hot path (arXiv 2111.06704).

The compute path is the C-ABI library ``libcpm.so`` (``include/cpm.h``) built from
``csrc/`` for sm_103a; ``paper_2111_06704_gb300.cpm`` is its thin ctypes binding.
Importing this package loads nothing; ``workloads`` only places atoms and ions.
"""
