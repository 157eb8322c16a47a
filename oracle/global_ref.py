"""Global assembly reference (test infrastructure): the sum over elements of
the element matrices at their global DOFs, by a library sparse sum (COO with
duplicates summed, then CSR with sorted columns)."""
import numpy as np


def assemble_csr(dofs, elem, nrows, upper=False):
    """(indptr, indices, data) of sum_e P_e^T A_e P_e for element matrices elem [E, n, n];
    upper=True: its upper triangle (columns >= row), the symmetric storage."""
    import scipy.sparse as sp
    d = np.asarray(dofs, dtype=np.int64)
    E, n = d.shape
    rows = np.repeat(d, n, axis=1).reshape(-1)
    cols = np.tile(d, (1, n)).reshape(-1)
    A = sp.coo_matrix((np.asarray(elem, dtype=np.float64).reshape(-1), (rows, cols)), shape=(nrows, nrows)).tocsr()
    A.sum_duplicates()
    if upper:
        A = sp.triu(A, k=0, format="csr")
    A.sort_indices()
    return A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data
