"""GB300-native low-synchronization block Arnoldi for restarted BFOM/BGMRES."""
